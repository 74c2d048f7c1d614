/*
 * xs_api.h -- C ABI of the GB300 direct-method XPCS / XSVS library (libxs.so).
 *
 * The library computes, on one GPU, the quantities of arXiv 2204.13241:
 *   - the scattered intensity I(q,t) = |S(q,t)|^2 with
 *     S(q,t) = sum_j f_j exp(+i q.r_j(t))            (Sec. 2.2, Eqs. pe_ri, Iq_pq;
 *     on reciprocal-lattice q = 2 pi h^-T n            Sec. 3.1, Eq. sq_cut_simple,
 *                                                     Algorithm 1),
 *   - the XPCS autocorrelation g2(q,tau)             (Sec. 2.3, Eq. g2_def),
 *   - the XSVS contrast of K-frame exposures         (Sec. 2.3, Eqs. inte_Iq, bq_Iq),
 *   - the gradient of a loss L(I) with respect to the atomic positions
 *     (the adjoint of Eq. pe_ri),
 * and, beyond that path: the intermediate scattering function and the
 * contrast it predicts (Eqs. Fq_pq, norm_Fq, beta_alt_int), intensities at
 * point lists and on the Ewald-sphere slice (Fig. 5), per-species
 * q-dependent form factors (Sec. 2.1), the FFT-based method (Sec. 3.2,
 * Algorithm 2) as a cross-check, and XSVS over pixel shards.
 * Sign convention: the paper writes p^e = sum f exp(-i q.r); this library's
 * amplitude S is its complex conjugate.  I, g2 and the contrast are identical.
 *
 * Conventions for every entry point
 *   - Units: positions and cell in Angstrom; q in 1/Angstrom; time in frames.
 *   - Cell: xs_box.h is the row-major 3x3 matrix whose COLUMNS are the cell
 *     edge vectors, so fractional coordinates are s = h^-1 r and the detector
 *     points are q = 2 pi h^-T n for integer Miller indices n.  A cubic box of
 *     side L is h = L * identity.
 *   - Grids: xs_qgrid gives n_x in [nx0, nx0+nx), n_y in [ny0, ny0+ny),
 *     n_z in [nz0, nz0+nz); pixel p = (iz*ny + iy)*nx + ix (x fastest).
 *   - Ownership: the caller owns every input and output buffer; the library
 *     never frees or retains them past the call.  Internal workspace is taken
 *     from the context's allocator and kept by the context for reuse.
 *   - Asynchrony: all GPU work is enqueued on the caller's CUDA stream
 *     (`cuda_stream`, a cudaStream_t; NULL = legacy default stream) and the
 *     call returns without waiting, except where host buffers are read or
 *     written (stated per call).
 *   - Errors: arguments are checked before any launch; a bad argument returns
 *     XS_ERR_INVALID_ARG and enqueues nothing.  Failures found by a kernel
 *     (a bounded wait that timed out, a non-finite position) set the
 *     context's device error word; xs_sync_status() reports it.  No C++
 *     exception crosses this ABI and no kernel traps.  xs_last_error() gives
 *     a message for the last non-OK status of the calling thread.
 */
#ifndef XS_API_H
#define XS_API_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define XS_API __attribute__((visibility("default")))
#else
#define XS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XS_OK = 0,
    XS_ERR_INVALID_ARG = 1,   /* null pointer, size <= 0, singular cell, tau/K out of range */
    XS_ERR_UNSUPPORTED = 2,   /* valid request this library does not implement */
    XS_ERR_NO_MEMORY = 3,     /* the allocator returned NULL */
    XS_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the CUDA error) */
    XS_ERR_TIMEOUT = 5,       /* a kernel's bounded wait expired (device error word) */
    XS_ERR_NUMERIC = 6,       /* a kernel met a non-finite input (device error word) */
    XS_ERR_BOUNDS = 7         /* a bounds check of the checked build failed (device error word; the
                                 access was skipped) */
} xs_status;

/* Arithmetic of the intensity (Sec. 3.1 direct method; every variant computes
 * the same S, they differ only in rounding):
 *   XS_PREC_FP32_DIRECT  one FP32 phase factor per atom and pixel from an exact
 *                        integer phase, FP32 sums merged in FP64 blocks;
 *   XS_PREC_SPLIT_FP16   tensor-core contraction over atoms of FP16 hi+lo split
 *                        factor tables, FP32 accumulation flushed per atom chunk;
 *   XS_PREC_SPLIT_BF16   the same with BF16 hi+lo tables;
 *   XS_PREC_FP32_FACTORED  the factorised sum on the FP32 pipes: per tile of
 *                        64 x 64 (n_x, n_y) and 32 atoms, tables E_x and
 *                        f E_z E_y of FP32 factors from exact integer phases,
 *                        one complex FMA per atom and pixel, 32-atom FP32
 *                        sums added into error-free FP32 pairs.  Same error
 *                        level as XS_PREC_FP32_DIRECT (<= 1e-6), about ten
 *                        times faster; xs_intensity and the batched calls only. */
typedef enum {
    XS_PREC_FP32_DIRECT = 0,
    XS_PREC_SPLIT_FP16 = 1,
    XS_PREC_SPLIT_BF16 = 2,
    XS_PREC_FP32_FACTORED = 3
} xs_precision;

typedef struct { double h[9]; } xs_box;                          /* row-major, columns = edges */
typedef struct { int32_t nx0, nx, ny0, ny, nz0, nz; } xs_qgrid;  /* Miller-index ranges */

/* One trajectory.  pos is float32 [n_frames][n_atoms][3] (unwrapped
 * coordinates are fine: the method is periodic, Sec. 3.1); on the device, or
 * in host memory when pos_on_host != 0 (then the library streams frames to the
 * device in chunks; page-locked memory lets the copies overlap compute).
 * f is float32 [n_atoms] in the same memory space as pos. */
typedef struct {
    const float* pos;
    int32_t pos_on_host;
    const float* f;
    int64_t n_atoms;
    int64_t n_frames;
    xs_box box;
} xs_traj;

/* Device-memory allocator used for workspace.  alloc returns NULL on
 * failure; free receives pointers alloc returned.  Both are called on the
 * calling host thread.  NULL allocator = cudaMalloc / cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} xs_allocator;

typedef struct xs_context xs_context;

/* Creates a context bound to the current CUDA device: workspace cache, tuned
 * tile choices and the device error word.  *out receives the handle. */
XS_API xs_status xs_context_create(const xs_allocator* allocator, xs_context** out);

/* Synchronizes the device, frees the workspace and the handle. NULL is a no-op. */
XS_API xs_status xs_context_destroy(xs_context* ctx);

/*
 * Intensity on a detector grid for every frame: Algorithm 1 of Sec. 3.1
 * (direct method), S(q,t) = sum_j f_j exp(+i q.r_j(t)), I = |S|^2 (Eq. Iq_pq).
 *   I_out   float32 [n_frames][nz][ny][nx]
 *   amp_out float32 [n_frames][nz][ny][nx][2] = (Re S, Im S), or NULL
 * Outputs may be device or host memory (detected per pointer); host outputs
 * make the call wait for the stream.  XS_PREC_SPLIT_* work in 128 x 128 tiles
 * of (n_x, n_y) per plane (a partial tile is computed whole and cut); any grid
 * size works with every precision.  With device outputs, the split path
 * contracts only half of a grid that is (nearly) symmetric under n -> -n when
 * that needs fewer tiles, and fills the rest by S(-q) = conj S(q), which holds
 * for the real form factors of this library: the half n_x <= 0 of a plane at
 * n_z = 0, or the planes n_z <= 0 of a volume (the other axes widened to the
 * hull of their range and its mirror).  A 192 x 192 centred plane takes 2
 * tiles instead of 4 and the volume [-40, 40]^3 41 instead of 81; the half
 * lives in the context workspace.
 */
XS_API xs_status xs_intensity(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid,
                       xs_precision prec, float* I_out, float* amp_out, void* cuda_stream);

/*
 * Many independent trajectories in one persistent launch (the batched form
 * of Algorithm 1).  traj[i], grid[i] and I_out[i] as in xs_intensity, with
 * device positions; n_traj >= 1.  `traj`, `grid` and `I_out` are host arrays.
 * Grids are contracted as halves filled by I(-q) = I(q) where that saves
 * tiles, as in xs_intensity (the intensity's pair form is a sum of
 * f_i f_j cos(q.r_ij), even in q for real form factors).  With the split
 * precisions, repeated calls with the same arguments replay one captured
 * CUDA graph.
 */
XS_API xs_status xs_intensity_batched(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid,
                               int32_t n_traj, xs_precision prec, float* const* I_out,
                               void* cuda_stream);

/*
 * The correlation stages requested for one trajectory of xs_xpcs_batched,
 * both of the trajectory's own intensity: g2 on its delays (Sec. 2.3 Eq.
 * g2_def, as xs_g2) and the XSVS contrast on its window lengths and |q| rings
 * (Sec. 2.3 Eqs. inte_Iq and bq_Iq, as xs_xsvs_contrast).  A stage whose count
 * (n_tau, or n_K or n_rings) is 0 is skipped.
 *   taus            host int32 [n_tau], each in [0, n_frames)
 *   g2_out          device float64 [n_tau][P], P = pixels of the trajectory's grid
 *   mean_out        device float64 [P], or NULL
 *   Ks              host int32 [n_K], each in [1, n_frames]
 *   ring_width      in (0, 1], in units of 2 pi / det(h)^(1/3); rings as in
 *                   xs_xsvs_contrast
 *   beta_out        device float64 [n_K][n_rings]
 *   ring_count_out  host int32 [n_rings] (pixels per ring, written during the
 *                   call), or NULL
 */
typedef struct {
    const int32_t* taus;
    int32_t n_tau;
    double* g2_out;
    double* mean_out;
    const int32_t* Ks;
    int32_t n_K;
    double ring_width;
    int32_t n_rings;
    double* beta_out;
    int32_t* ring_count_out;
} xs_corr_request;

/*
 * The batched pipeline of the direct method: the intensities of many
 * trajectories as in xs_intensity_batched (Algorithm 1, Sec. 3.1), then each
 * trajectory's g2 and XSVS contrast as requested in req[i] (a host array of
 * n_traj requests; Sec. 2.3).  With the split precisions every kernel of the
 * call -- the phase records, the one persistent contraction over all
 * trajectories, the mirror fills and, trajectory after trajectory, the g2 and
 * XSVS kernels -- is captured into one CUDA graph on the first call and
 * replayed by later calls with the same arguments.  The correlation stages of
 * the trajectories share one region of the context workspace and run in
 * order.  Invalid requests (a delay or window length out of range, a missing
 * output) return XS_ERR_INVALID_ARG before anything is launched.
 */
XS_API xs_status xs_xpcs_batched(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, int32_t n_traj,
                                 xs_precision prec, float* const* I_out, const xs_corr_request* req,
                                 void* cuda_stream);

/*
 * The paper's FFT-based method (Sec. 3.2, Algorithm 2), as a cross-check of the
 * direct method: each atom's Gaussian (standard deviation eta, in A) is added
 * on the k nearest grid points per axis of an n_grid^3 grid over the
 * orthorhombic cell (periodic), the grid is Fourier transformed (FFT kernels
 * of this library, FP64), and p^eta is divided by the transform of one
 * truncated Gaussian at the origin; I = |p^e|^2 on `grid`.  The method's own
 * errors (grid aliasing, cut-off) are small when eta spans about two grid
 * steps and the cut-off +-5 eta.
 *   n_grid   power of two in [8, 1024]; Miller indices of `grid` must lie in
 *            [-n_grid/2, n_grid/2)
 *   k_cut    grid points per axis around each atom (<= 64), or <= 0 for the
 *            smallest integer above 10 eta in grid steps
 *   I_out    device float32 [T][nz][ny][nx]; amp_out device [...][2] or NULL
 * Uses n_grid^3 complex FP64 of context workspace; frames run one by one.
 */
XS_API xs_status xs_intensity_fft(xs_context* ctx, const xs_traj* traj, int32_t n_grid, double eta, int32_t k_cut,
                                  const xs_qgrid* grid, float* I_out, float* amp_out, void* cuda_stream);

/*
 * Intensity at an arbitrary list of reciprocal-lattice points n (Miller
 * indices), I(n,t) = |sum_j f_j exp(+i q.r_j(t))|^2 with q = 2 pi h^-T n (the
 * same sum as xs_intensity; Sec. 3.1, Algorithm 1 over a pixel set that is not
 * a box, such as the Ewald-sphere slice of xs_ewald_points).
 *   XS_PREC_FP32_DIRECT   the FP32 direct kernel on the points
 *   XS_PREC_SPLIT_*       the points are grouped by n_z; every 128 x 128 tile
 *                         of a plane's bounding box that holds a point goes
 *                         through the tensor-core kernel (one batched launch)
 *                         and the points are gathered from the tiles
 *   miller   HOST int32 [P][3]
 *   traj     device positions (pos_on_host = 0)
 *   I_out    device float32 [T][P]; amp_out device float32 [T][P][2] or NULL
 * Uses context workspace for the records and, on the tensor path, the tiles.
 */
XS_API xs_status xs_intensity_points(xs_context* ctx, const xs_traj* traj, const int32_t* miller, int64_t P,
                                     xs_precision prec, float* I_out, float* amp_out, void* cuda_stream);

/*
 * Host-side helper (no GPU work): the detector slice on the Ewald sphere
 * (Fig. 5: |k_f| = |k_i| with k_f = k_i + q) as reciprocal-lattice points.
 * For each (n_x, n_y) of the window, q(n_z) = 2 pi h^-T (n_x, n_y, n_z) is a
 * line that meets the sphere |q + k_in| = |k_in| where A n_z^2 + B n_z + C = 0;
 * the root nearer n_z = 0 is kept and, of the two integers around it, the one
 * whose q lies nearer the sphere (ties: the smaller |n_z|).
 *   k_in        incident wave vector, 1/A (|k_in| = 2 pi / lambda)
 *   miller_out  HOST int32 [nx*ny][3], x fastest; n_z = 0 where invalid
 *   valid_out   HOST uint8 [nx*ny] (1: the line meets the sphere), or NULL
 */
XS_API xs_status xs_ewald_points(const xs_box* box, const double* k_in, int32_t nx0, int32_t nx, int32_t ny0,
                                 int32_t ny, int32_t* miller_out, uint8_t* valid_out);

/*
 * Intensity with q-dependent form factors of several atom species (Sec. 2.1:
 * f_i(q), each species' form factor a sum of Gaussians in |q|):
 *   S(q,t) = sum_j f_j F_{s_j}(q) exp(+i q.r_j(t)),   I = |S|^2,
 *   F_s(q) = sum_{k<4} a_k exp(-b_k (|q|/4 pi)^2) + c,
 * with f_j = traj->f[j] a per-atom weight (1 for plain species; 0 drops an
 * atom, as for tracer labelling).  Each species runs through the phase and
 * contraction kernels of xs_intensity on its own atoms; the per-species
 * amplitudes are combined in FP64.
 *   traj      device positions (pos_on_host = 0) and device weights f [N]
 *   species   HOST int32 [N], values in [0, n_species)
 *   coef      HOST float64 [n_species][9] = (a1, b1, a2, b2, a3, b3, a4, b4, c),
 *             b in A^2 (|q| in 1/A)
 *   I_out     device float32 [T][nz][ny][nx]; amp_out device float32 [...][2] or NULL
 * Uses context workspace for one species' records and three per-frame buffers.
 */
XS_API xs_status xs_intensity_species(xs_context* ctx, const xs_traj* traj, const int32_t* species,
                                      int32_t n_species, const double* coef, const xs_qgrid* grid,
                                      xs_precision prec, float* I_out, float* amp_out, void* cuda_stream);

/*
 * XPCS autocorrelation, Sec. 2.3 Eq. g2_def, per pixel:
 *   mean(p) = (1/T) sum_{t<T} I(t,p)
 *   g2(tau,p) = [(1/(T-tau)) sum_{t<T-tau} I(t,p) I(t+tau,p)] / mean(p)^2
 *   I        device float32 [T][P]
 *   taus     HOST int32 [n_tau], each 0 <= tau < T (tau = 0 gives beta_0 + 1,
 *            Eq. bq_g2)
 *   g2_out   device float64 [n_tau][P]; NaN or Inf where mean(p) == 0
 *   mean_out device float64 [P], or NULL
 */
XS_API xs_status xs_g2(xs_context* ctx, const float* I, int64_t T, int64_t P, const int32_t* taus,
                int32_t n_tau, double* g2_out, double* mean_out, void* cuda_stream);

/*
 * XSVS contrast, Sec. 2.3 Eqs. inte_Iq and bq_Iq, averaged over exposures:
 * for each window length K, exposures I_K(p,w) = sum_{t=wK}^{wK+K-1} I(t,p),
 * w = 0..floor(T/K)-1; ring r (1..n_rings) holds the pixels with
 * r - ring_width/2 <= |q|/Delta < r + ring_width/2, Delta = 2 pi / det(h)^(1/3);
 *   beta_K(r) = mean_w [ (<I_K^2>_r - <I_K>_r^2) / <I_K>_r^2 ]  (population variance).
 *   I              device float32 [T][P] on `grid` (P = nx*ny*nz)
 *   Ks             HOST int32 [n_K], 1 <= K <= T
 *   ring_width     in units of Delta, 0 < ring_width <= 1
 *   beta_out       device float64 [n_K][n_rings]; NaN for an empty ring
 *   ring_count_out HOST int32 [n_rings] pixels per ring, or NULL
 */
XS_API xs_status xs_xsvs_contrast(xs_context* ctx, const float* I, int64_t T, const xs_qgrid* grid,
                           const xs_box* box, const int32_t* Ks, int32_t n_K, double ring_width,
                           int32_t n_rings, double* beta_out, int32_t* ring_count_out,
                           void* cuda_stream);

/*
 * Intermediate scattering function from the amplitudes, Sec. 2.3 Eqs. Fq_pq
 * and norm_Fq.  The paper's p^e is the conjugate of the amplitude S returned
 * by xs_intensity, so
 *   F(tau,p)    = [(1/(T-tau)) sum_{t<T-tau} conj(S(t,p)) S(t+tau,p)] / sum_f2
 *   F_hat(tau,p) = F(tau,p) / F(0,p),  F(0,p) = [(1/T) sum_{t<T} |S(t,p)|^2] / sum_f2
 *   amp       device float32 [T][P][2] (re, im), as written by xs_intensity
 *   taus      HOST int32 [n_tau], each 0 <= tau < T
 *   sum_f2    sum_j f_j^2 of the atoms (> 0)
 *   F_out     device float64 [n_tau][P][2]
 *   Fhat_out  device float64 [n_tau][P][2], or NULL; NaN where F(0,p) == 0
 */
XS_API xs_status xs_isf(xs_context* ctx, const float* amp, int64_t T, int64_t P, const int32_t* taus,
                        int32_t n_tau, double sum_f2, double* F_out, double* Fhat_out, void* cuda_stream);

/*
 * Contrast predicted from F_hat through the Siegert relation, Sec. 2.3 Eq.
 * beta_alt_int, in the form that matches exposures summing K frames (as in
 * xs_xsvs_contrast):
 *   ratio_K(r) = mean over the pixels p of ring r of
 *                (1/K^2) sum_{i,j<K} |F_hat(|i-j|,p)|^2,   |F_hat(0,p)|^2 = 1,
 * i.e. beta_K(r) / beta_0(r).  Rings as in xs_xsvs_contrast.
 *   Fhat           device float64 [Kmax][P][2] for the delays 0..Kmax-1 (row 0
 *                  is not read)
 *   Ks             HOST int32 [n_K], 1 <= K <= Kmax, any order (NULL if n_K == 0)
 *   ratio_out      device float64 [n_K][n_rings]; NaN for an empty ring (NULL
 *                  allowed when n_K or n_rings is 0)
 *   ring_count_out HOST int32 [n_rings] pixels per ring, or NULL
 * Uses n_K * (pixels in rings) float64 of context workspace.
 */
XS_API xs_status xs_contrast_from_isf(xs_context* ctx, const double* Fhat, int64_t Kmax, const xs_qgrid* grid,
                                      const xs_box* box, const int32_t* Ks, int32_t n_K, double ring_width,
                                      int32_t n_rings, double* ratio_out, int32_t* ring_count_out,
                                      void* cuda_stream);

/*
 * XSVS over pixel shards (one GPU per shard): the sums that the contrast of
 * xs_xsvs_contrast is made of, for the shard's pixels.  For window length
 * Ks[k] and window w (0 <= w < T / Ks[k]) the row is kw = sum_{k'<k} T / Ks[k']
 * + w, and
 *   sums_out[kw][r - 1] = (sum_p I_K(p,w), sum_p I_K(p,w)^2) over the pixels p
 *   of the shard in ring r,   I_K(p,w) = sum_{t=wK}^{wK+K-1} I(t,p)
 * Adding the shards' sums and counts (an all-reduce) and passing them to
 * xs_xsvs_finalize gives the contrast of all pixels.
 *   I          device float32 [T][P] (the shard's pixels)
 *   ring       HOST int32 [P]: ring of each pixel, 1..n_rings, 0 for none (as
 *              from xs_ring_index on the full grid)
 *   sums_out   device float64 [n_kw][n_rings][2]
 *   count_out  HOST int64 [n_rings] pixels per ring in the shard, or NULL
 */
XS_API xs_status xs_xsvs_partial(xs_context* ctx, const float* I, int64_t T, int64_t P, const int32_t* ring,
                                 int32_t n_rings, const int32_t* Ks, int32_t n_K, double* sums_out,
                                 int64_t* count_out, void* cuda_stream);

/*
 * Host-side (no GPU work): beta_K(r) from summed shard sums and counts (HOST
 * arrays laid out as in xs_xsvs_partial), with the per-window contrast of Eq.
 * bq_Iq averaged over windows; NaN for an empty ring.  beta_out HOST float64
 * [n_K][n_rings].
 */
XS_API xs_status xs_xsvs_finalize(const double* sums, const int64_t* counts, int64_t T, const int32_t* Ks,
                                  int32_t n_K, int32_t n_rings, double* beta_out);

/*
 * Host-side helper (no GPU work): the ring of every pixel of `grid` as used by
 * xs_xsvs_contrast, ring_out HOST int32 [nx*ny*nz], 0 for pixels in no ring.
 */
XS_API xs_status xs_ring_index(const xs_qgrid* grid, const xs_box* box, double ring_width, int32_t n_rings,
                        int32_t* ring_out);

/*
 * Adjoint of the intensity for one frame (traj->n_frames must be 1, device
 * positions):  dL/dr_j = sum_q dL/dI_q * 2 Re[ conj(S_q) * i q f_j exp(i q.r_j) ].
 *   amp        device float32 [P][2], the S of this frame (xs_intensity amp_out)
 *   dL_dI      device float32 [P]
 *   dL_dr_out  device float32 [n_atoms][3]
 * The contraction over n_y runs on tensor cores in split BF16 (FP32
 * accumulation; relative error near 1e-5), the rest in FP32; every grid shape
 * is accepted.  Uses context workspace for the tensor-core images of
 * H = dL/dI conj(S) (32 B per pixel, with (n_x, n_z) rows rounded up to 64
 * and n_y to 32) and per-atom partial sums (12 B per atom and 64 rows).
 */
XS_API xs_status xs_intensity_backward(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid,
                                const float* amp, const float* dL_dI, float* dL_dr_out,
                                void* cuda_stream);

/* Autotuner of the tensor-core path (no counterpart in the paper: Algorithm 1
 * does not depend on how the q grid is tiled).  Times, on up to 64 frames of
 * `traj` (device positions) on `grid`, every tile kind -- 128 n_x x 128 n_y
 * (tile_kind 0) and 128 n_x x 64 n_y (tile_kind 1; not for grids contracted
 * as a half, which are planned on 128 x 128 tiles) -- with FP32 accumulation
 * chunks of 16, 32 and 64 stages of 64 atoms, and keeps the fastest pair in
 * the context under the trajectory's shape bucket: atom count rounded down to
 * a power of two (after padding to a multiple of 64), grid extents and
 * precision.  Later xs_intensity calls, and every trajectory of later
 * batched calls, whose bucket matches use it; untuned shapes take tile kind 1
 * when the grid's n_y extent is at most 64 (the same number of tiles), else
 * tile kind 0, with 64-stage chunks.  Synchronizes the stream. */
XS_API xs_status xs_tune(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, xs_precision prec,
                  void* cuda_stream);

/* The tile kind (0: 128 x 128, 1: 128 x 64) and chunk length (stages of 64
 * atoms) that the split precisions use for n_atoms atoms on `grid`: the
 * tuned choice of the shape bucket (see xs_tune), else the default rule.
 * Host only; launches nothing. */
XS_API xs_status xs_tuned_choice(xs_context* ctx, int64_t n_atoms, const xs_qgrid* grid, xs_precision prec,
                                 int32_t* tile_kind, int32_t* chunk_stages);

/* Message for the last non-OK status returned on the calling thread. */
XS_API const char* xs_last_error(void);

/* Waits for `cuda_stream`, then reads and clears the device error word:
 * XS_ERR_TIMEOUT, XS_ERR_NUMERIC, XS_ERR_BOUNDS (checked build only) or
 * XS_OK. */
XS_API xs_status xs_sync_status(xs_context* ctx, void* cuda_stream);

/* Table builder of the split-precision (tensor-core) paths, a test and
 * measurement option of this library (Sec. 3.1 fixes only what the tables
 * hold, exp(i 2 pi n s) per atom and index).  mode 0 (the default): each
 * producer thread evaluates a seed exp(i 2 pi n0 U / 2^32) and
 * exp(i 2 pi U / 2^32) of exact 32-bit turn counts U in FP32 and advances
 * along n by complex multiplication; mode 1: every entry is sincospi of its
 * exact turn count n U mod 2^32 in FP64, rounded once to FP32 (and the B
 * side's weight f E_z in FP64), which makes the contraction several times
 * slower.  The choice holds for later calls on the context. */
XS_API xs_status xs_set_table_builder(xs_context* ctx, int32_t mode);

/* Debug knob: the bounded waits inside the tensor-core kernel give up after
 * `ns` nanoseconds (default 2e9).  Used by tests to force a timeout on a
 * kernel whose wait can never complete. */
XS_API xs_status xs_set_wait_timeout_ns(xs_context* ctx, int64_t ns);

/* Tracing.  When enabled, every kernel launch of the context is bracketed by
 * CUDA events recorded on the launching stream.  xs_profile_read waits for
 * those events and returns, for launch groups whose name starts with `prefix`
 * ("" = all), the summed device time in milliseconds and the number of
 * kernels since the last read, and forgets those records (others stay).  Launch groups: "phase"
 * (phase records, 1 kernel), "direct" (FP32 direct sum, 1-2), "factored" (factorised FP32 sum, 1-2), "tc"
 * (tensor-core contraction, 1), "split_finish" (pieces of the last wave, 1),
 * "friedel" (fill of a half grid, 1), "g2" (2), "xsvs" (segment totals,
 * prefix, windows, finalize: 1-4), "isf" (1), "isf_contrast" (2), "species"
 * (form-factor table, per-species sum, finish: 1 each), "points" (gather,
 * 1), "fft" (spread, three line passes, gather: 4-5), "batched"
 * (graph replay: its kernels), "adjoint" (4).  xs_launch_count returns the
 * number of kernels the context has launched since it was created (tracing
 * on or off). */
XS_API xs_status xs_profile_enable(xs_context* ctx, int32_t on);
XS_API xs_status xs_profile_read(xs_context* ctx, const char* prefix, double* total_ms, int64_t* launches);
XS_API xs_status xs_launch_count(xs_context* ctx, int64_t* count);

/*
 * The FP32 direct-sum intensity of xs_intensity(..., XS_PREC_FP32_DIRECT, ...)
 * (the same kernels and the same result) for callers that cannot allocate
 * device memory when they need it: real-time or embedded hosts that fix their
 * device memory budget at start-up, plug-ins running inside an application
 * that owns the device memory, and processes whose framework allocator
 * already holds the whole device.  The paper has no counterpart: this is a
 * service of the library, not a step of the method.
 *   - No context and no allocation: the scratch (phase records, T * ceil64(N)
 *     * 16 bytes, plus the partial amplitudes of the atom splits) lives in one
 *     static device array of 16 MiB that every GPU loading the library keeps
 *     until the process exits.  Requests needing more are rejected with
 *     XS_ERR_INVALID_ARG and a message giving the bytes needed and available.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     with the target device current); the lookup enqueues no work, and a
 *     device reset or another context on the device cannot leave a stale
 *     address behind.  The first call on a device may load the library's
 *     device code there: make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents (each
 *     call writes every byte it reads).  Calls whose kernels overlap on the
 *     GPU (unordered streams) race on it.
 *   - traj->pos, traj->f, I_out and amp_out (nullable) are device memory laid
 *     out as for xs_intensity; dev_err is an optional caller-owned device int
 *     that the kernels OR with 2 when a position or form factor is not finite.
 *   - Argument checks are those of xs_intensity: grid extents up to 65,536,
 *     at most 2^31 atoms and 65,535 frames, and every pointer the kernels use
 *     must be device (or managed) memory; anything else returns
 *     XS_ERR_INVALID_ARG before a kernel is launched.
 */
XS_API xs_status xs_intensity_fp32_static(const xs_traj* traj, const xs_qgrid* grid, float* I_out,
                                          float* amp_out, int* dev_err, void* cuda_stream);

/* Library version string. */
XS_API const char* xs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XS_API_H */
