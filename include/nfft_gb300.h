/*
 * nfft_gb300.h -- C ABI of the GB300 (sm_103a) NFFT window-convolution library.
 *
 * The library computes the nonequispaced fast Fourier transform of
 * arXiv 2208.00049 (NFFT.jl), Sec. 2.2:
 *
 *   direct  (Algorithm 1):  fhat = B F D f      fhat_j ~ sum_{n in I_N} f_n e^{-2 pi i n.k_j}
 *   adjoint (Algorithm 2):  y    = D^T F^H B^T fhat   y_n ~ sum_j fhat_j e^{+2 pi i n.k_j}
 *
 * with D the resampling correction (deconvolution) plus zero pad / crop,
 * F the FFT on the sigma-oversampled grid (cuFFT), and B the sparse
 * window-resampling matrix (Eq. Bmatrix) built from a Kaiser-Bessel window
 * truncated to [-m, m) grid cells (2m points per dimension, Sec. 3.7.5).
 *
 * Conventions (all entry points):
 *  - Arrays are row-major (C order).  f and y have shape (N_1, ..., N_D) with
 *    array index i_d = n_d + floor(N_d/2) for n in I_N (Sec. 2.1).  Nodes k
 *    have shape (M, D), k[j][d] in [-1/2, 1/2) (values outside are wrapped
 *    periodically).  fhat has M entries in the caller's node order.
 *  - Complex values are interleaved (re, im): complex64 (NFFT_C64) or
 *    complex128 (NFFT_C128).  The plan's dtype fixes the real type of every
 *    buffer except k, whose type is given to nfft_set_nodes.
 *  - Buffers are owned by the caller and must be contiguous.  Pointers may be
 *    device pointers (the call is then asynchronous on the plan's stream) or
 *    host pointers (pageable or pinned); with a host pointer the library
 *    stages the data through plan-owned device memory and the call returns
 *    only once host outputs are written.
 *  - The plan owns the oversampled grid, the sorted node records, the
 *    deconvolution vectors, the cuFFT plan and all scratch memory.
 *  - Every entry point returns an int status: NFFT_OK (0) or a negative
 *    NFFT_ERR_* code.  No C++ exception crosses the ABI.  A failure inside a
 *    CUDA or cuFFT call is latched in the plan (sticky) and returned by every
 *    later call on that plan until it is destroyed.
 */
#ifndef NFFT_GB300_H
#define NFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define NFFT_OK                 0
#define NFFT_ERR_INVALID_ARG   -1   /* argument out of range, null pointer, bad shape */
#define NFFT_ERR_NO_NODES      -2   /* a transform was requested before nfft_set_nodes */
#define NFFT_ERR_OOM           -3   /* device allocation failed */
#define NFFT_ERR_CUFFT         -4   /* cuFFT returned an error */
#define NFFT_ERR_CUDA          -5   /* CUDA runtime returned an error */
#define NFFT_ERR_TIMEOUT       -6   /* a bounded device wait gave up */
#define NFFT_ERR_DEVICE_CHECK  -7   /* a device-side range check failed (reserved: no
                                        kernel of this build makes such checks) */
#define NFFT_ERR_UNSUPPORTED   -8   /* valid but not supported by this build */

/* ---- dtypes and flags ------------------------------------------------ */
#define NFFT_C64   0   /* complex64 data, FP32 resampling, FP32 accumulation */
#define NFFT_C128  1   /* complex128 data, FP64 everywhere */

/* Support [-m, m] instead of [-m, m): nodes exactly on a grid line get the
   extra tap at u = +m, i.e. the (2m+1)^D footprint discussed in Sec. 3.7.5. */
#define NFFT_FLAG_CLOSED_SUPPORT  0x1u
/* FP32 scatter with compensated summation: every accumulator (a register of
   the 2D and 3D complex64 kernels, a shared-memory tile element of the
   generic kernels) also accumulates the rounding error of each addition
   (TwoSum) and adds it back at the flush. */
#define NFFT_FLAG_COMPENSATED     0x2u
/* FULL precomputation (Sec. 3.7.4 item 2; the paper's GPU prototype of
   Sec. 6): nfft_set_nodes also builds the sparse matrix B of Eq. Bmatrix
   ((2m)^D values and column indices per node) and its transpose, and the
   resampling steps apply them with cuSPARSE SpMM instead of the tiled
   kernels.  A comparison form: it stores and moves far more than the grid.
   NFFT_ERR_UNSUPPORTED when M (2m)^D >= 2^31 or D = 3 with m > 6. */
#define NFFT_FLAG_FULL_MATRIX     0x4u
/* (2m+2)^D footprint with the untruncated window (continued past |u| = m
   by its sin form): the NFFT3 variant discussed in Sec. 3.7.5, slightly more
   accurate than 2m points at the same m (Sec. 5.1).  Exclusive with
   NFFT_FLAG_CLOSED_SUPPORT. */
#define NFFT_FLAG_WIDE_WINDOW     0x8u
/* Run the correction + zero-pad + FFT steps of Algorithm 1 and the inverse
   FFT + crop + correction steps of Algorithm 2 as the separate correction
   kernels around a full cuFFT transform even where the plan
   qualifies for the pruned FFT or the direct sums (see nfft_step_pad_fft). */
#define NFFT_FLAG_LIBRARY_FFT     0x10u

/* Window values (Sec. 3.7.4).  Without these flags complex64 plans use the
   specialised 2D and 3D kernels where they apply (window from its
   POLYNOMIAL representation), complex128 plans with m >= 7 or an
   oversampling of at least 1.5 (and half-open support) a POLYNOMIAL window
   fitted in FP64 at degree max(2m, 16), whose fit error is at the FP64
   rounding level (about 1e-14 of the window peak), and every other plan the
   window evaluated.  Each flag below selects the generic kernels (any D, m, dtype)
   with one way of obtaining the window values, so that the three can be
   compared on the same kernels; at most one may be given:
     DIRECT      the window evaluated per tap (sinh, sqrt);
     LINEAR      the lookup table psi_s = psi_Base(s/(S-2)), s < S,
                 S = m 2^{c_min(m,8)} + 2 with NFFT3's c = (3, 7, 9, 14, 17,
                 20, 23, 24), read with linear interpolation (Eq. linInterp);
                 built in FP64 at plan creation, one table per dimension in
                 the plan's real type (m = 8: 1.3e8 entries per dimension);
                 not with NFFT_FLAG_WIDE_WINDOW; NFFT_ERR_UNSUPPORTED beyond
                 8 GB of tables;
     POLYNOMIAL  per-tap polynomials of degree 2m (Chebyshev interpolation
                 in FP64) evaluated by Horner; not with
                 NFFT_FLAG_CLOSED_SUPPORT or NFFT_FLAG_WIDE_WINDOW.
   None of them with NFFT_FLAG_FULL_MATRIX. */
#define NFFT_FLAG_WINDOW_DIRECT     0x20u
#define NFFT_FLAG_WINDOW_LINEAR     0x40u
#define NFFT_FLAG_WINDOW_POLYNOMIAL 0x80u

typedef struct nfft_plan nfft_plan;

/* ---- plan ------------------------------------------------------------- */

/* Create a plan (Sec. 3.1-3.2: the plan allocates every temporary and does
 * the precomputation).
 *   out    : receives the plan; *out is NULL on failure.
 *   D      : dimension, 1..3.
 *   N      : N[0..D-1], each >= 2 (even or odd).
 *   M      : number of nodes, >= 0 (0 gives empty transforms).
 *   sigma  : oversampling factor > 1; N~_d = sigma N_d rounded up to even.
 *   m      : window half-width, 1..10 (1..8 for D = 3: NFFT_ERR_UNSUPPORTED
 *            beyond), with 2m < N~_d.
 *   dtype  : NFFT_C64 or NFFT_C128.
 *   flags  : NFFT_FLAG_* bits.
 *   stream : cudaStream_t on which every later call enqueues its work
 *            (NULL = legacy default stream).
 * Precomputation done here on the device, in FP64 (Sec. 3.5): the
 * deconvolution vectors beta_d(n_d) = 1/I0(m sqrt(b^2 - (2 pi n_d/N~_d)^2)),
 * b = pi (2 - N_d/N~_d).  The current CUDA device becomes the plan's device.
 */
int nfft_plan_create(nfft_plan **out, int D, const int64_t *N, int64_t M,
                     double sigma, int m, int dtype, uint32_t flags,
                     void *stream);

/* Release everything the plan owns.  NULL is accepted. */
int nfft_plan_destroy(nfft_plan *p);

/* Set the nodes (Sec. 3.7.3: nodes are grouped by the grid block R_p they
 * fall in).  k: (M, D) array, FP64 if k_is_fp64 != 0 else FP32 (for either
 * plan dtype; FP32 nodes are promoted to FP64), host or device.  In FP64,
 * x = N~_d k_{j,d} is split into the cell floor(x) mod N~_d and the fraction
 * x - floor(x) (rounded to the plan's real type); nodes are bin-sorted by
 * grid tile on the device.  The library copies what it needs: the caller
 * may free k on return (device k: once the stream reaches this call). */
int nfft_set_nodes(nfft_plan *p, const void *k, int k_is_fp64);

/* Direct NFFT, Algorithm 1: fhat = B F D f.  f: N_1 x ... x N_D complex,
 * fhat: M complex. */
int nfft_forward(nfft_plan *p, const void *f, void *fhat);

/* Adjoint NFFT, Algorithm 2: y = D^T F^H B^T fhat.  fhat: M complex,
 * y: N_1 x ... x N_D complex. */
int nfft_adjoint(nfft_plan *p, const void *fhat, void *y);

/* Node gradient through the direct NFFT (the paper defines none; this is
 * the derivative of Eq. SumOverNode with respect to k_{j,d}):
 *   gk[j][d] = Re( conj(cot_j) * d fhat_j / d k_{j,d} ),
 *   d fhat_j / d k_{j,d} = N~_d sum_l ghat_l psi'(u_d) prod_{e != d} psi(u_e),
 * ghat = F D f.  cot: M complex (the upstream gradient of a real loss with
 * respect to fhat, PyTorch convention); gk: (M, D) real of the plan's real
 * type.  The same call gives the node gradient of y = A^H w for upstream Y
 * with f := Y and cot := w. */
int nfft_grad(nfft_plan *p, const void *f, const void *cot, void *gk);

/* Block the host until all work enqueued by this plan has finished; returns
 * the first error seen.  Errors found on the device surface here: the 3D
 * complex64 m = 4 gather and node gradient copy a tile region with the
 * tensor memory accelerator and wait for it on a shared-memory barrier
 * with an iteration limit; a copy that never arrives makes the kernel
 * return early and this call return NFFT_ERR_TIMEOUT (the outputs of that
 * transform are then undefined).  The flag behind it is kept per device,
 * not per plan: the first nfft_plan_sync after the event, of any plan on
 * that device that uses these kernels, reports it and clears it. */
int nfft_plan_sync(nfft_plan *p);

/* Static, human-readable text for a status code. */
const char *nfft_strerror(int code);

/* ---- introspection and the individual steps ---------------------------
 * The transforms above are compositions of these steps; they are exported
 * so that each step can be timed and checked on its own.  All take device
 * pointers and run asynchronously on the plan's stream. */

/* N~ (oversampled sizes), the tile shape in grid cells, and the number of
 * work items of the current node set (0 before nfft_set_nodes; reading it
 * synchronises the plan's stream). */
int nfft_plan_info(nfft_plan *p, int64_t *Ntilde3, int64_t *tile3, int64_t *n_items);

/* Device pointer to the plan's oversampled grid (N~_1 x ... x N~_D complex,
 * natural FFT order: grid index l is stored at position l mod N~). */
void *nfft_plan_grid(nfft_plan *p);

/* Choose the tile shape (grid cells per tile per dimension) used by the
 * resampling kernels; takes effect at the next nfft_set_nodes.  Used by the
 * autotuner.  Tiles must satisfy 1 <= tile_d <= N~_d and fit the shared
 * memory limit with their halo.  The tile also selects the kernels (see
 * nfft_plan_paths): the specialised complex64 ones need tiles of at most
 * 9 cells per dimension (3D m = 4; the gather also accepts larger tiles in
 * dimensions 0 and 1), 5 (3D m = 6) or 9 x 25 (2D m = 4); other tiles run the
 * generic kernels.  Defaults: 9 x 9 x 8 (3D m = 4), 5 x 5 x 5 (3D m = 6),
 * 9 x 25 or 8 x 8 (2D m = 4, by grid size), 20 x 20 (2D complex128, m = 8)
 * or 16 x 16 (2D complex128, m <= 6), else a power-of-two cube sized for the
 * node density. */
int nfft_plan_set_tile(nfft_plan *p, const int64_t *tile3);

/* Algorithm 1, correction and zero-pad step: resampling correction and zero
 * pad of f into the plan grid (fftshift folded into the index map,
 * Sec. 3.5). */
int nfft_step_deconv_pad(nfft_plan *p, const void *f);

/* The FFT step of Algorithm 1 (sign = -1, cuFFT FORWARD) or the inverse FFT
 * step of Algorithm 2 (sign = +1, cuFFT INVERSE, unnormalised), in place on
 * the plan grid. */
int nfft_step_fft(nfft_plan *p, int sign);

/* Algorithm 1, resampling step (Algorithm 3): block-partitioned resampling
 * (gather) from the plan grid to fhat (M complex, caller order). */
int nfft_step_gather(nfft_plan *p, void *fhat);

/* Algorithm 2, adjoint resampling step (Algorithm 4): block-partitioned
 * adjoint resampling (scatter) of fhat onto the plan grid; the grid is
 * cleared first. */
int nfft_step_scatter(nfft_plan *p, const void *fhat);

/* Algorithm 2, crop and correction step: crop of the plan grid to I_N and
 * resampling correction into y. */
int nfft_step_crop_deconv(nfft_plan *p, void *y);

/* Algorithm 1, correction + zero-pad + FFT steps in one call: correction,
 * zero pad and forward FFT of f into the plan grid (the grid then holds
 * ghat as after
 * nfft_step_deconv_pad + nfft_step_fft(-1)).  For D = 3, complex64 and
 * N~_d = 2 N_d = 256 (and without NFFT_FLAG_LIBRARY_FFT) this is the pruned
 * FFT: three passes of 256-point line DFTs that read only the non-zero part
 * of the padded grid, with the correction fused into the first pass and the
 * fftshift of Sec. 3.5 applied as the exact phase i^l (N~ = 2N).  For small
 * 1D complex128 plans (see nfft_plan_paths) it is the direct sum
 * g^_l = sum_n f_n beta(n) e^{-2 pi i n l / N~} over the N inputs.
 * Otherwise it runs the two separate steps. */
int nfft_step_pad_fft(nfft_plan *p, const void *f);

/* Algorithm 2, inverse FFT + crop + correction steps in one call:
 * unnormalised inverse FFT of the plan grid, crop to I_N and correction into
 * y.  Pruned as for nfft_step_pad_fft
 * (each inverse pass computes only the N outputs that are kept; the plan
 * grid is used as scratch and does not hold the full inverse FFT
 * afterwards), as direct sums for small 1D complex128 plans;
 * otherwise nfft_step_fft(+1) + nfft_step_crop_deconv. */
int nfft_step_fft_crop(nfft_plan *p, void *y);

/* Graph mode for small transforms, whose time is mostly kernel launches:
 * with enable != 0, nfft_forward and nfft_adjoint called with device
 * buffers are captured into a CUDA graph (on an internal stream) the first
 * time a pair of buffers is seen and replayed on the plan's stream with one
 * launch afterwards; new buffers re-capture, and nfft_plan_set_tile drops the
 * graphs (nfft_set_nodes keeps them: the node buffers stay in place).  Host
 * buffers, and plans with NFFT_FLAG_FULL_MATRIX (whose matrices are
 * reallocated by nfft_set_nodes), take the direct path.  enable = 0 drops
 * the graphs.  Returns NFFT_ERR_INVALID_ARG for a null plan and a latched
 * error of the plan if it holds one. */
int nfft_plan_set_graph(nfft_plan *p, int enable);

/* Asynchronous host-buffer transforms: with enable != 0, nfft_forward and
 * nfft_adjoint called with a HOST input and a HOST output return as soon as
 * the work is enqueued: the input is copied to a plan-owned device buffer on
 * a copy stream, the transform runs on the plan's stream, the result is
 * copied back on a second copy stream, and the three are ordered by events.
 * Two sets of device buffers alternate between calls, so consecutive calls
 * overlap one call's copies with the previous call's kernels.  The host
 * buffers must stay valid (inputs unchanged, outputs unread) until
 * nfft_plan_sync returns, which waits for all three streams; page-locked
 * host memory (cudaHostAlloc, torch pin_memory) is needed for the copies to
 * overlap.  Calls with a device input or output keep the synchronous
 * behaviour described at nfft_forward.  enable = 0 waits for the copy
 * streams and restores it.  Returns NFFT_ERR_INVALID_ARG for a null plan and
 * a latched error of the plan if it holds one. */
int nfft_plan_set_async(nfft_plan *p, int enable);

/* Which kernels the plan's transforms use (set by nfft_plan_create and
 * nfft_plan_set_tile): *fast_resample bit 0 = a specialised complex64
 * gather (3D m = 4 or 6, 2D m = 4), bit 1 = a register-accumulating
 * complex64 scatter (3D m = 4 or 6 with tiles of at most 17 - 2m cells per
 * dimension, 2D m = 4); *pruned_fft = how nfft_step_pad_fft /
 * nfft_step_fft_crop run: 0 = library FFT with separate correction steps,
 * 1 = the pruned 3D FFT, 2 = direct sums (1D complex128 with N~ <= 4096 and
 * N N~ <= 2^20: the FFT's definition evaluated over the N non-zero inputs or
 * kept outputs, spread over every SM, for sizes where one library FFT would
 * occupy a single SM's FP64 units).  Either pointer may be NULL. */
int nfft_plan_paths(nfft_plan *p, int *fast_resample, int *pruned_fft);

/* Node-gradient resampling on the current plan grid (which must hold
 * ghat = F D f): gk[j][d] = Re(conj(cot_j) d fhat_j / d k_{j,d}). */
int nfft_step_grad_gather(nfft_plan *p, const void *cot, void *gk);

/* Tile-shape autotuner.  The paper sweeps the block size (Sec. 5.2) and
 * proposes choosing it automatically by measurement, like FFTW_MEASURE
 * (Sec. 6): for each candidate tile this times forward + adjoint on the
 * given nodes (k as for nfft_set_nodes), keeps the fastest, caches the
 * choice per (device, D, N, M, sigma, m, dtype, flags) for the process, and
 * leaves the plan with that tile and the nodes set.  chosen3 (may be NULL)
 * receives the tile.  Allocates temporary device buffers; synchronises. */
int nfft_plan_autotune(nfft_plan *p, const void *k, int k_is_fp64, int64_t *chosen3);

/* ---- batched transforms -------------------------------------------------
 * Many independent problems of one dimension D, sigma, m and dtype, with
 * uneven sizes, run as one persistent gather / scatter launch over all their
 * work items, one deconvolution launch, and one batched cuFFT per distinct
 * oversampled size (Algorithms 1 and 2 applied to each problem); the size
 * classes' FFTs run concurrently on internal streams forked from and joined
 * back to `stream`.
 *   B problems; problem p has coefficient size N[p*D .. p*D+D-1] and uses
 *   node set set_of[p] (0 <= set_of[p] < S).  S node sets, set s has
 *   M_set[s] nodes; problems sharing a node set must have equal N (several
 *   right-hand sides on one set).  Every set must be used.
 * Buffers are device pointers to concatenations, in order:
 *   k    : node sets in set order, each (M_set[s], D), FP64 if k_is_fp64;
 *   f, y : problems in problem order, each N_p row-major complex;
 *   fhat : problems in problem order, each M_set[set_of[p]] complex.
 * All calls are asynchronous on `stream` except nfft_batch_set_nodes and
 * nfft_batch_autotune, which synchronise.  Status codes as above. */
typedef struct nfft_batch nfft_batch;
int nfft_batch_create(nfft_batch **out, int D, int B, const int64_t *N, const int32_t *set_of, int S,
                      const int64_t *M_set, double sigma, int m, int dtype, uint32_t flags,
                      void *stream);
int nfft_batch_destroy(nfft_batch *b);
int nfft_batch_set_nodes(nfft_batch *b, const void *k, int k_is_fp64);
int nfft_batch_forward(nfft_batch *b, const void *f, void *fhat);
int nfft_batch_adjoint(nfft_batch *b, const void *fhat, void *y);
/* Graph mode: each direction is captured once into a CUDA graph (on an
 * internal stream) and replayed on `stream` while the buffers passed stay
 * the same; new buffers trigger a re-capture. */
int nfft_batch_set_graph(nfft_batch *b, int enable);
/* Common tile shape (cells per dimension, clamped per problem); discards the
 * node sort (call nfft_batch_set_nodes again). */
int nfft_batch_set_tile(nfft_batch *b, const int64_t *tile3);
/* Tile shape, total work items (0 before set_nodes; synchronises) and the
 * number of distinct oversampled sizes (one cuFFT plan each). */
int nfft_batch_info(nfft_batch *b, int64_t *tile3, int64_t *n_items, int64_t *n_fft_classes);
/* Autotuner for a batch: as nfft_plan_autotune, timing the whole batch. */
int nfft_batch_autotune(nfft_batch *b, const void *k, int k_is_fp64, int64_t *chosen3);

/* ---- spreading without device allocation ------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not call cudaMalloc: code living under another framework's
 * allocator (a raw cudaMalloc beside a caching allocator fragments memory
 * and may synchronise the device), latency-critical loops that cannot take
 * the implicit device synchronisation of cudaMalloc / cudaFree, and services
 * whose device memory must be reserved when the library loads.
 *
 * It spreads nodes onto the oversampled grid without a plan (complex64,
 * half-open support, 2m taps per dimension):
 *   grid[l] = sum_j fhat_j prod_d w_d(N~_d k_{j,d} - l_d),
 * with the Kaiser-Bessel window scaled to 1 at u = 0 (the same quantity
 * nfft_step_scatter leaves in a plan's grid).  grid is N~_1 x ... x N~_D
 * complex64 in natural FFT order, N~_d = sigma N_d rounded up to even; it is
 * overwritten.  k: (M, D) FP64, fhat: M complex64; all three are device
 * pointers owned by the caller, on the current device (memory of another
 * device is rejected); the call is asynchronous on `stream`.
 *
 * Scratch: the bin-sort buffers live in one static device array sized for
 * M <= NFFT_NOALLOC_MAX_NODES nodes and at most NFFT_NOALLOC_MAX_TILES
 * tiles (about 11 MB, held on every GPU that loads the library until the
 * process exits).  Larger sizes return NFFT_ERR_UNSUPPORTED; invalid
 * arguments or host pointers return NFFT_ERR_INVALID_ARG.  Nothing is
 * allocated: no cudaMalloc, no cudaFree, no allocating library routine.
 * The array is shared by all calls on a device and keeps the last call's
 * contents (each call clears what must start at zero); calls that overlap on
 * the GPU race on it and must be serialised by the caller.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it, so make that first call before any stream capture, and do
 * not use this call across a device reset (cudaDeviceReset), after which the
 * cached address is stale. */
#define NFFT_NOALLOC_MAX_NODES  262144
#define NFFT_NOALLOC_MAX_TILES  65536
int nfft_spread_noalloc(int D, const int64_t *N, double sigma, int m, int64_t M,
                        const double *k, const void *fhat, void *grid, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NFFT_GB300_H */
