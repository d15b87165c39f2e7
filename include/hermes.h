/*
 * hermes.h -- C ABI of the B300 field-window estimator (libhermes.so).
 *
 * The library computes the paper's in-situ clustering statistics on one GPU:
 *   (a) a weighted catalogue is projected onto an N^3 periodic grid of order-p
 *       B-spline scaling functions (Eq. phi_projection, Sec. 3.1);
 *   (b) the density contrast is Fourier transformed (Sec. 2 convention);
 *   (c) the spectrum is multiplied by shell windows K = W^ Phi^ (Sec. 3.5, the
 *       K_W equation) -- plain shells (Eq. Wshell_k), Legendre-weighted shells
 *       (Sec. 3.4.3) and Y_lm-weighted shells (Eq. multipole-window) -- and
 *       inverse transformed;
 *   (d) the filtered fields are contracted cell by cell into xi(r), xi_l(s) and
 *       zeta_l(r1, r2) (Eq. pair-counting, Eq. 2rdEs, Eq. 2-fold-translation),
 *       normalised as Delta DD / RR with analytic uniform randoms
 *       (Eq. xi-deltaDD-over-RR).
 *
 * Conventions common to every entry point:
 *   - Every function returns a status: HERMES_OK (0) or a negative HERMES_ERR_*.
 *     Nothing aborts and no C++ exception crosses the ABI.  After an error,
 *     hermes_last_error() describes it.
 *   - Output arrays are host float64 arrays owned and sized by the caller.
 *   - Input pointers are only read during the call; the caller keeps ownership.
 *   - A context owns all device memory it uses, lives on the CUDA device that
 *     was current when it was created, and restores the caller's current device
 *     before returning.  A context must not be used by two host threads at once;
 *     distinct contexts are independent.
 *   - Calls are synchronous with respect to their results: when a function that
 *     writes a host output returns HERMES_OK, the output is complete.
 */
#ifndef HERMES_H
#define HERMES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HERMES_OK 0
#define HERMES_ERR_ARG (-1)     /* invalid argument (null, size, value)            */
#define HERMES_ERR_RANGE (-2)   /* data outside the accepted range (positions, r)  */
#define HERMES_ERR_NOMEM (-3)   /* device or host allocation failed                */
#define HERMES_ERR_CUDA (-4)    /* a CUDA runtime call failed                      */
#define HERMES_ERR_TIMEOUT (-5) /* a bounded device wait gave up                   */
#define HERMES_ERR_STATE (-6)   /* call out of order (e.g. xi before assign)       */

/* flags of hermes_assign */
#define HERMES_DEVICE_PTR 1u /* pos / w are device pointers on the context's GPU   */
#define HERMES_WRAP 2u       /* wrap coordinates periodically instead of rejecting */
#define HERMES_EAGER 4u      /* batched calls: launch directly, no CUDA graph       */

typedef struct hermes_ctx hermes_ctx;

/*
 * Create a context for a periodic box of side L, N = 2^j cells per axis and an
 * order-p centred B-spline basis (p = 4 is cubic).  N = 2^J follows the MRA
 * resolution level of Sec. 4.1 (task.J, "L = 2**J grid cells per axis").
 *   L > 0; 4 <= j <= 10 and N == 1 << j; 1 <= p <= 8 and 2p - 1 <= N.
 * Allocates the resident field (N^3 float32) and its half spectrum.
 * Errors: HERMES_ERR_ARG on a bad value, HERMES_ERR_NOMEM, HERMES_ERR_CUDA.
 * *out is set to NULL on error.
 */
int hermes_create(double L, int N, int p, int j, hermes_ctx **out);

/* Free every resource of the context.  NULL is accepted (no-op). */
int hermes_destroy(hermes_ctx *ctx);

/*
 * Run all later work of the context on `cuda_stream` (a cudaStream_t of the
 * context's device), or on the context's own stream when NULL.
 */
int hermes_set_stream(hermes_ctx *ctx, void *cuda_stream);

/*
 * Project a weighted catalogue onto the grid, Eq. (phi_projection):
 *   eps_l = sum_i w_i prod_d M_p(u_{i,d} - l_d),
 * then form delta = eps / eps_bar - 1 with eps_bar = sum w / N^3 and transform
 * it (delta^(0) := 0).  The result replaces the resident field; it is reused by
 * every later statistic until the next hermes_assign.
 *   pos : n x 3 float32, row-major (x, y, z), in [0, L).  Index rule: u =
 *         fl32(x * fl32(N/L)); a coordinate is accepted when 0 <= u <= N, or,
 *         with HERMES_WRAP, when |u| < 2^22 (cells are then taken modulo N).
 *   w   : n float32 weights (marks, masses, ...), or NULL for unit weights.
 *   n   : number of points, n >= 1.
 *   flags: HERMES_DEVICE_PTR when pos / w are device memory of the context's
 *         device (e.g. torch tensor data pointers), HERMES_WRAP as above.
 * Errors: HERMES_ERR_ARG (null pointer, n < 1, a device flag on a non-device
 * pointer), HERMES_ERR_RANGE (a rejected coordinate, a non-finite weight, or
 * sum w <= 0; the resident field is then invalid), HERMES_ERR_NOMEM,
 * HERMES_ERR_CUDA.
 */
int hermes_assign(hermes_ctx *ctx, const float *pos, const float *w, int64_t n, unsigned flags);

/*
 * hermes_assign for callers that cannot allocate GPU memory at call time.  Some
 * hosts own all device memory through an allocator of their own (a framework's
 * caching pool that has reserved most of the GPU, an embedding application with a
 * fixed memory budget): a cudaMalloc behind their back may fail or push them out
 * of memory, and a cudaFree waits for the whole device, stalling every stream of
 * the host.  Others run a serving loop whose latency must not include allocator
 * calls.  This entry point does what hermes_assign does, with the same arguments
 * and errors, but calls no cudaMalloc, cudaFree or other allocating routine.
 * (The paper has no counterpart; this is an interface of this library only.)
 *   - pos / w must already be device memory of the context's device (no host
 *     staging copy); HERMES_DEVICE_PTR is implied, HERMES_WRAP is honoured.
 *   - The block partial sums of the weight and self-pair reductions use one
 *     fixed 256 KiB array in device memory (32768 float64), which every GPU
 *     that loads the library keeps until the process exits.  The context order p
 *     must satisfy 2 + max(2, p^3) * 148 <= 32768, i.e. p <= 6; a larger p is
 *     rejected with HERMES_ERR_ARG and a message naming the limit.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress), which may load the library's device code; make
 *     that first call before any stream capture begins.
 *   - Every call on a device shares the array: calls whose work overlaps on the
 *     GPU (other contexts on other streams included) race on it; serialise them.
 *     Each call overwrites every entry it reads, so no state carries over.
 *   - Like hermes_assign, the call waits for the context's stream twice (it reads
 *     the range flag and the weight sums on the host before the transform).
 * The context must have been created (hermes_create allocates the field).
 */
int hermes_assign_noalloc(hermes_ctx *ctx, const float *pos, const float *w, int64_t n, unsigned flags);

/*
 * Define the radial bins [r_edges[b], r_edges[b+1]) of every later statistic
 * and tabulate, in float64 on the host, the r^2-weighted bin average of the
 * spherical Bessel functions <j_l>_b(k) for 0 <= l <= l_max at every discrete
 * |k| of the grid (Eq. Wshell_k for l = 0; Sec. 3.4.3, "its average over the
 * corresponding radial window", for l > 0).  Tables are stored as float32.
 *   r_edges: strictly increasing, r_edges[0] >= 0, r_edges[n_edges-1] <= L/2.
 *   n_edges: 2 .. 4097.   l_max: 0 .. 24.
 * Errors: HERMES_ERR_ARG, HERMES_ERR_RANGE (edges out of range), HERMES_ERR_NOMEM.
 */
int hermes_window_shells(hermes_ctx *ctx, const double *r_edges, int n_edges, int l_max);

/*
 * Isotropic 2PCF xi(r_b) of the resident field for every bin (Landy-Szalay
 * Delta DD / RR with uniform randoms, Eq. xi-deltaDD-over-RR):
 *   xi_b = (1/N^3) sum_x delta(x) delta~_b(x) - SN_b,
 * delta~_b = iFFT[delta^ W^_b Phi^], W^_b the volume-normalised finite shell
 * (Eq. Wshell_k), Phi^(n) = prod_d sinc^{2p}(pi n_d / N); SN_b is the exact
 * self-pair term sum_i w_i^2 K_eff,b(x_i, x_i) / (N^3 eps_bar^2).
 *   out: n_bins float64.
 * Errors: HERMES_ERR_STATE (no field or no bins), HERMES_ERR_ARG, HERMES_ERR_CUDA.
 */
int hermes_xi(hermes_ctx *ctx, double *out);

/*
 * Legendre multipoles xi_l(s_b) with the line of sight along +z, kernel
 * (2l+1) i^l <j_l>_b(k) L_l(k_z/k) Phi^ (Sec. 3.4.3), normalised like xi
 * (RR_0 = 1 in delta units), self-pair term subtracted.
 *   ells: n_ells even orders, each 0 <= l <= l_max of the current bins
 *         (odd orders vanish identically for an auto-correlation).
 *   out : [n_ells][n_bins] float64.  ells[i] == 0 reproduces hermes_xi.
 * Errors: HERMES_ERR_STATE, HERMES_ERR_ARG, HERMES_ERR_CUDA.
 */
int hermes_xi_multipoles(hermes_ctx *ctx, const int *ells, int n_ells, double *out);

/*
 * The same statistics as hermes_xi_multipoles, evaluated in Fourier space by
 * Parseval's theorem (Eq. pair-counting-kspace): one pass over the half spectrum
 * accumulates, per order l, the float64 histogram over |n|^2 of
 * w_z Phi^(n) L_l(k_z/k) (|delta^_n|^2 - S^(n)/eps_bar^2), then
 * xi_{b,l} = (2l+1) i^l sum_q <j_l>_b(q) A_l(q) / N^6.  No inverse transform is
 * run, so the cost is one read of delta^ for all windows.  The self-pair term is
 * subtracted exactly as in hermes_xi_multipoles; the results agree to rounding.
 *   ells: 1..8 even orders <= l_max; out: [n_ells][n_bins] float64.
 * Errors: as hermes_xi_multipoles.
 */
int hermes_xi_multipoles_kspace(hermes_ctx *ctx, const int *ells, int n_ells, double *out);

/*
 * xi_l of many catalogues in one call (the estimator of Eq. 2rdEs and its
 * multipole form, Sec. 3, applied to each catalogue separately): catalogue k is
 * points [offsets[k], offsets[k+1]) of pos (n x 3 float32) and w (n float32 or
 * NULL = unit weights), gridded on this context's N^3 grid and measured with
 * its shells.  Each catalogue gets its own mean density, self-pair table and
 * fields; the context's single resident field (hermes_assign) is untouched.
 * Every pass runs as one launch over a chunk of catalogues; the whole
 * measurement is captured into a CUDA graph on the context's stream and
 * replayed by later calls of the same shape (same n_cat, total points, weights
 * present or not, orders and plan); HERMES_EAGER (or the legacy default stream)
 * launches the same kernels directly instead.
 *   offsets: host array of n_cat + 1 int64, offsets[0] = 0, strictly increasing
 *            (no empty catalogue); n = offsets[n_cat].
 *   n_cat:   1..1024.  ells: 1..8 even orders <= l_max.
 *   flags:   HERMES_DEVICE_PTR (pos, w are device memory of this device),
 *            HERMES_WRAP, HERMES_EAGER.  Inputs are copied into the context
 *            during the call.
 *   out:     [n_cat][n_ells][n_bins] float64, host.
 * Windows per launch S and catalogues per launch C come from
 * hermes_batch_set_plan, else from a process-wide cache for this shape, else
 * from timing candidates on the first call (the autotuner).
 * Errors: as hermes_assign and hermes_xi_multipoles; HERMES_ERR_RANGE names the
 * catalogue whose weights do not sum to a positive number.
 */
int hermes_xi_multipoles_batch(hermes_ctx *ctx, const float *pos, const float *w, const int64_t *offsets,
                               int n_cat, const int *ells, int n_ells, unsigned flags, double *out);

/*
 * Fixes the batch plan: S windows per launch (multiple of 4, <= 32) and C
 * catalogues per launch (1..1024); S = C = 0 returns to autotuning.
 * Errors: HERMES_ERR_ARG.
 */
int hermes_batch_set_plan(hermes_ctx *ctx, int S, int C);

/*
 * The plan of the last batched call and its graph: S, C, kernels in the graph,
 * graph replays so far, and the autotuner's timings as triples
 * {S, C, ms per catalogue-window} (up to tune_cap triples; *n_tune = count).
 * Any pointer may be NULL.  Errors: HERMES_ERR_ARG.
 */
int hermes_batch_info(hermes_ctx *ctx, int *S, int *C, int64_t *graph_kernels, int64_t *graph_replays,
                      double *tune, int tune_cap, int *n_tune);

/*
 * Density-dependent marks (Sec. 3.3, Eq. power-law-mark, Eq. inverse-density-mark).
 * The resident field is smoothed with a window (HERMES_SMOOTH_SPHERE: Table A1 row
 * (b), radius R; HERMES_SMOOTH_GAUSS: row (c), width R), K = W^ Phi^, and read back
 * at each of the n positions through the same basis as the scatter (its adjoint):
 *   rho_i = 1 + sum_l phi_l(x_i) delta~_l,  delta~ = iFT(delta^ K),
 * the smoothed density in units of the mean sum w / L^3 (it equals
 * sum_j w_j K_eff(x_i, x_j) / eps_bar).  With remove_self, one object per window
 * volume (4 pi R^3 / 3, or (2 pi)^{3/2} R^3) is subtracted, r = max(rho - self, 0):
 *   HERMES_MARK_DENSITY   out_i = rho_i
 *   HERMES_MARK_POWER     out_i = (r + b)^a        (b the regulariser epsilon, a = alpha)
 *   HERMES_MARK_INVERSE   out_i = ((b + 1) / (b + r))^a  (b = rho_* / rho_bar, a = p).
 * Pass the marks to hermes_assign as weights for the marked statistics.
 *   pos: n x 3 float32 (host, or device with HERMES_DEVICE_PTR, like out: n float32).
 * Errors: HERMES_ERR_ARG, HERMES_ERR_RANGE (bad R or a coordinate outside [0, L]),
 * HERMES_ERR_STATE (no field, or explicit randoms set), HERMES_ERR_CUDA, HERMES_ERR_NOMEM.
 */
#define HERMES_SMOOTH_SPHERE 0
#define HERMES_SMOOTH_GAUSS 1
#define HERMES_MARK_DENSITY 0
#define HERMES_MARK_POWER 1
#define HERMES_MARK_INVERSE 2
int hermes_density_marks(hermes_ctx *ctx, int window, double R, int kind, double a, double b, int remove_self,
                         const float *pos, int64_t n, unsigned flags, float *out);

/*
 * Explicit random catalogue for the Landy-Szalay estimator in the field language
 * (Sec. 3.3, Eq. xi-deltaDD-over-RR): xi[W] = Delta DD[W] / RR[W] with
 * Delta = D - alpha R, alpha = sum w_D / sum w_R, both fields in units of the mean
 * data density, and the self pairs of D and R removed from both products.
 * The random field, its transform (k = 0 mode kept) and its self-pair table stay
 * on the device; the next hermes_assign builds Delta from the data and them, and
 * hermes_xi / hermes_xi_multipoles / hermes_xi_cylinders (and the k-space forms)
 * then divide by RR (xi_l by the RR of the l = 0 window of each bin; RR by
 * Parseval on the random field).  Without randoms RR = 1 (analytic uniform randoms).
 * Arguments as hermes_assign.  Invalidates the resident field (assign the data
 * again).  zeta_l and hermes_assign_noalloc refuse to run while randoms are set
 * (HERMES_ERR_STATE); batched calls use analytic randoms.
 * Errors: as hermes_assign.
 */
int hermes_assign_randoms(hermes_ctx *ctx, const float *pos, const float *w, int64_t n, unsigned flags);
/* Back to analytic uniform randoms (invalidates a resident difference field). */
int hermes_clear_randoms(hermes_ctx *ctx);

/*
 * Axisymmetric windows for the redshift-space 2PCF xi(r_perp, r_par), line of
 * sight z (Sec. 3.4.4, the finite-bin ring window; Table A1 rows (f)-(i)):
 *   K_{j,i}(n) = <J_0(k_perp rho)>_i exp(-k_perp^2 sigma_perp^2 / 2)
 *                * <cos(k_par z)>_j * Phi^(n),
 * <J_0>_i the area average over the annulus perp_edges[i] <= rho < perp_edges[i+1]
 * (a first edge 0 gives the disk 2 J_1(kR)/(kR)), <cos>_j the average over the slab
 * pair par_edges[j] <= |z| < par_edges[j+1] (a first edge 0 gives the filled slab
 * sin(kH)/(kH)); sigma_perp > 0 multiplies the Gaussian transverse smoothing of
 * the Gaussian ring.  Tables are built on the host in float64 (closed forms with
 * J_1) and stored on the device as float32, indexed exactly by
 * q_perp = n_x^2 + n_y^2 and |n_z|.  Replaces earlier cylindrical bins.
 *   edges: 2..4097 per axis, >= 0, strictly increasing, <= L/2.
 * Errors: HERMES_ERR_ARG, HERMES_ERR_RANGE, HERMES_ERR_NOMEM, HERMES_ERR_CUDA.
 */
int hermes_window_cylinders(hermes_ctx *ctx, const double *perp_edges, int n_perp_edges, const double *par_edges,
                            int n_par_edges, double sigma_perp);

/*
 * xi(r_perp, r_par) of the resident field with the cylindrical bins: the window
 * multiply, inverse transforms and cell contraction of hermes_xi_multipoles with
 * K_{j,i}, minus the exact self-pair term, normalised by the uniform RR (= 1 in
 * delta units, K(0) = 1).  out: [n_par][n_perp] float64.
 * Errors: HERMES_ERR_STATE (no field or no cylindrical bins), HERMES_ERR_TIMEOUT,
 * HERMES_ERR_CUDA, HERMES_ERR_NOMEM.
 */
int hermes_xi_cylinders(hermes_ctx *ctx, double *out);

/* The same by Parseval's theorem (Eq. pair-counting-kspace): one pass over delta^
 * histograms (|delta^|^2 - S^/eps_bar^2) Phi^ <cos>_j over q_perp, contracted with
 * the transverse table.  Errors: as hermes_xi_cylinders. */
int hermes_xi_cylinders_kspace(hermes_ctx *ctx, double *out);

/*
 * Ring windows for the redshift-space 2PCF at a list of (r_perp, r_par) points, such
 * as the (s, mu) samples r_perp = s sqrt(1 - mu^2), r_par = s mu of xi(s, mu)
 * (Sec. 3.4.4, the circular-ring window; Table A1 row (i), "standard (s, mu)
 * binning geometry"), line of sight z.  Window w is
 *   K_w(n) = T_perp,w(k_perp) exp(-k_perp^2 sigma_perp^2 / 2) T_par,w(k_par) Phi^(n):
 *   dR_w = 0:  T_perp = J_0(k_perp R_w)            (thin ring)
 *   dR_w > 0:  T_perp = area average of J_0(k_perp rho) over max(0, R_w - dR_w/2) <= rho <= R_w + dR_w/2
 *   dH_w = 0:  T_par  = cos(k_par H_w)             (the double ring at z = +-H_w)
 *   dH_w > 0:  T_par  = average of cos(k_par z) over max(0, H_w - dH_w/2) <= |z| <= H_w + dH_w/2
 *              (sin(k dH/2)/(k dH/2) cos(k H) when the bin stays above 0).
 * Tables are built on the host in float64 (J_0, J_1 closed forms) and stored as
 * float32, indexed exactly by q_perp = n_x^2 + n_y^2 and |n_z|.  Replaces earlier
 * cylindrical bins (hermes_window_cylinders) and is replaced by them.
 *   R, H:   n values each, >= 0.   dR, dH: n widths each (>= 0), or NULL for 0 (thin).
 *   R + dR/2 <= L/2 and H + dH/2 <= L/2 for every window; n: 1..4096.
 * Errors: HERMES_ERR_ARG, HERMES_ERR_RANGE, HERMES_ERR_NOMEM, HERMES_ERR_CUDA.
 */
int hermes_window_rings(hermes_ctx *ctx, const double *R, const double *H, const double *dR, const double *dH,
                        int n, double sigma_perp);

/*
 * xi of the resident field for every ring window: window multiply, inverse
 * transforms and cell contraction (windows in batches, each with its own
 * line-of-sight factor), minus the exact self-pair term, over RR (uniform: 1;
 * explicit randoms: their ring-window RR).  out: n float64.
 * Errors: HERMES_ERR_STATE (no field or no ring windows), HERMES_ERR_TIMEOUT,
 * HERMES_ERR_CUDA, HERMES_ERR_NOMEM.
 */
int hermes_xi_rings(hermes_ctx *ctx, double *out);

/* The same by Parseval's theorem (Eq. pair-counting-kspace): per window, a histogram
 * over q_perp of (|delta^|^2 - S^/eps_bar^2) Phi^ T_par,w (eight windows per pass over
 * delta^), contracted with the window's transverse column.  Errors: as hermes_xi_rings. */
int hermes_xi_rings_kspace(hermes_ctx *ctx, double *out);

/*
 * 3PCF Legendre multipoles zeta_l(r_b1, r_b2), 0 <= l <= l_max, from the
 * harmonic shell fields a_{b,lm} = iFFT[delta^ 4 pi i^l <j_l>_b Y_lm Phi^]
 * (Eq. multipole-window, Eq. iFFT-multipoleSFC):
 *   zeta_l(b1,b2) = 1/(4 pi N^3) sum_x delta(x) sum_{m=-l}^{l} conj(a_{b1,lm}) a_{b2,lm},
 * so that zeta(r1, r2, theta) = sum_l zeta_l L_l(cos theta)
 * (Eq. 2-fold-translation).  Only m >= 0 fields are built; m < 0 follows by
 * conjugation.  Returned raw: the diagonal b1 == b2 includes self triplets.
 *   out: [l_max+1][n_bins][n_bins] float64 (symmetric in b1, b2).
 * Up to 16 bins are transformed and contracted together.  More bins are taken
 * in blocks of 8, and every pair of blocks runs as one batch of at most 16 bins
 * (B (B + 1) / 2 batches for B blocks, each Gram entry kept from its own pair).
 * Errors: HERMES_ERR_STATE, HERMES_ERR_ARG, HERMES_ERR_NOMEM, HERMES_ERR_CUDA,
 * HERMES_ERR_TIMEOUT (a bounded wait gave up).
 */
int hermes_zeta_multipoles(hermes_ctx *ctx, double *out);

/*
 * 3PCF monopole by triple connection coefficients (Eq. 3pcfddd, Eq. 2-fold-density,
 * Eq. 3PCF-ddd-monopole, Eq. con-coeff, Eq. DDD-vector-product) on the order-p
 * B-spline basis of the context:
 *   DDD(b1, b2) = (1/N^3) sum_l delta_l sum_{a,b} Gamma_{a,b} f_b1(l + a) f_b2(l + b),
 *   Gamma_{a,b} = int phi(u) phi(u - a) phi(u - b) du   (grid units, unit-integral phi),
 * with f_b = iFFT[delta^ <j_0>_b Phi^] the l = 0 shell-filtered coefficients of the
 * bins set by hermes_window_shells.  This is (1/N^3) int D F_b1 F_b2 du, the box
 * integral of the three spline fields, evaluated exactly by a Gauss-Legendre rule of
 * (3p - 1) / 2 points per axis in every knot cell (the integrand is a polynomial of
 * degree 3(p - 1) there).  With Gamma replaced by the identity stencil it is the cell
 * sum zeta_0 of hermes_zeta_multipoles; the two differ by the basis smoothing.
 * Returned raw (self triplets included), like zeta_l.
 *   out: [n_bins][n_bins] float64, symmetric.  Up to 16 bins form one Gram; more run
 *   every pair of 8-bin blocks (B (B + 1) / 2 runs for B blocks).
 * Device memory: min(n_bins, 16) half spectra and 2 (n_bins + 1) real fields of N^3.
 * Orders: the context's p must be 1 .. 4 (the sample kernels are built for those).
 * Errors: HERMES_ERR_ARG (out NULL, or p > 4), HERMES_ERR_STATE (no field, no bins,
 * explicit randoms set), HERMES_ERR_NOMEM, HERMES_ERR_CUDA.
 */
int hermes_ddd_monopole(hermes_ctx *ctx, double *out);

/* Text of the last error of this context (never NULL; empty after success). */
const char *hermes_last_error(const hermes_ctx *ctx);

/* ---- tracing (per-kernel device time; not in the paper, which reports stage times only) ---- */

/*
 * Enable (on != 0) or disable per-launch timing.  While enabled, every kernel
 * launch of the context is bracketed by CUDA events recorded on the launching
 * stream.  Enabling or disabling clears the accumulated totals.
 */
int hermes_trace_enable(hermes_ctx *ctx, int on);

/*
 * Per kernel class k (0 <= k < n, see hermes_kernel_name): accumulated device
 * milliseconds and launch counts since the last enable/read; then clears them.
 * Synchronises the context's stream.  Returns the number of kernel classes (>= 0)
 * or an error status.  ms / launches may be NULL.
 */
int hermes_trace_read(hermes_ctx *ctx, double *ms, int64_t *launches, int n);

/* Name of kernel class k ("" when out of range). */
const char *hermes_kernel_name(int k);

/* Total kernels this context has launched since it was created (-1 for NULL). */
int64_t hermes_launch_count(const hermes_ctx *ctx);

/* ---- inspection hooks (tests and tools; not needed for measurements) ---- */

/* Copy the resident real field delta (N^3 float32, z fastest) to the host. */
int hermes_debug_get_delta(hermes_ctx *ctx, float *host_out);

/* Copy the resident half spectrum delta^ (N x N x N/2 complex64, k_z in [0, N/2)). */
int hermes_debug_get_spectrum(hermes_ctx *ctx, float *host_out);

/*
 * Replace the resident field by a given real delta (N^3 float32 host array),
 * transform it, and set eps_bar = 1 with an empty self-pair table (planted-field
 * tests: xi then equals the plain contraction (1/N^3) sum delta delta~).
 */
int hermes_debug_set_delta(hermes_ctx *ctx, const float *host_delta);

/*
 * The device node rule for n points (host arrays): first[i*3+d] = index of the
 * first supporting node along axis d (mod N; -1 for a rejected coordinate) and
 * wts[(i*3+d)*p + o] = M_p(u - node_o), o = 0..p-1.  Allocates temporary device
 * memory.  HERMES_WRAP in flags as for hermes_assign.
 */
int hermes_debug_nodes(hermes_ctx *ctx, const float *pos, int64_t n, unsigned flags, int *first, float *wts);

/*
 * Failure-detection check of the bounded device waits (no counterpart in the
 * paper).  Runs a one-thread kernel that waits, with the same bounded mbarrier
 * wait that guards every bulk-copy pipeline, on a barrier phase that nothing
 * completes and for which no copy is issued.  The wait gives up after one second
 * of wall time, the kernel records it in the context's error word and exits, and
 * the call returns HERMES_ERR_TIMEOUT.  The context stays usable afterwards.
 */
int hermes_debug_bounded_wait(hermes_ctx *ctx);

/*
 * Failure-detection hook for allocation errors (no counterpart in the paper):
 * the next `count` device allocations made by the library, in any context of
 * this process, report out of memory without allocating (count <= 0 disarms).
 * The failing call returns HERMES_ERR_NOMEM and keeps what it held before.
 * Returns the previous count.  No device is needed.
 */
int hermes_debug_fail_allocs(int count);

/* sums[0] = sum w, sums[1] = sum w^2, and the p^3 self-pair table (float64). */
int hermes_debug_get_sums(hermes_ctx *ctx, double *sums2, double *selfpair_p3);

/*
 * Host-only (no GPU needed): the float64 bin-averaged Bessel table the context
 * would upload, out[((b*(l_max+1)) + l)*Q + q] for q = |n|^2 in [0, Q),
 * Q = 3 (N/2 - 1)^2 + 1, k_q = 2 pi sqrt(q) / L.
 */
int hermes_shell_table_host(double L, int N, const double *r_edges, int n_edges, int l_max, double *out);

/* Number of table entries Q for a grid of N cells per axis. */
int64_t hermes_shell_table_len(int N);

/*
 * Frees the context's transient device buffers: the window work buffer, the
 * harmonic fields of zeta_l, the staging buffers of host inputs and the scatter's
 * per-point scratch.  The resident field, its spectrum, the window tables and
 * explicit randoms stay, so every later statistic still runs (re-growing what it
 * needs).  Waits for the context's stream.  (No counterpart in the paper: memory
 * management for long-lived contexts, used by the request server when a context
 * changes statistic.)  Errors: HERMES_ERR_ARG, HERMES_ERR_CUDA.
 */
int hermes_release_buffers(hermes_ctx *ctx);

/* ------------------------------------------------------------------------
 * FFT pass variants and their autotuner.  (The transforms are those of Sec. 3.5;
 * how a pass is tiled on the GPU has no counterpart in the paper.)
 *
 * pass: the three inverse passes of the xi statistics: HERMES_PASS_WINDOW, the
 * first (along x, window multiply fused in); HERMES_PASS_INV_Y, the inverse
 * transform along y of every filtered window; HERMES_PASS_CONTRACT, the last
 * (complex-to-real along z fused with the cell contraction); and
 * HERMES_PASS_ZETA_Y, the inverse transform along y of the zeta_l harmonic fields
 * (tuned on the first field of the first zeta_l call, before the x pass writes it);
 * HERMES_PASS_ZETA_X / HERMES_PASS_ZETA_X_M0, the first zeta_l pass (along x, the Y_lm
 * window multiply fused in) for complex fields / for the packed real m = 0 fields.
 * A variant fixes
 *   kind: inverse y: 0 the radix-8 pass, 1 one tile per block, 2 persistent blocks;
 *         window:    0 one window at a time, 1 two windows in flight per thread, 2 the
 *                    k_y and N - k_y lines together;
 *         contract:  0 the radix-8 pass, 1 16 values per thread;
 *         zeta y:    0 the radix-8 pass, 1 one tile per block;
 *         zeta x:    0 one line set at a time, 2 the k_y and N - k_y lines together;
 *   E:    values per thread (8: radix-8 stages; 16, 32: radix-16 or radix-32
 *         stages, fewer shared-memory exchanges per line for more registers);
 *   W:    tile width, the adjacent k_z columns one block transforms together
 *         (1 for the contraction pass, whose z lines are contiguous);
 *   minb: blocks per SM the kernel is compiled for (0: not fixed).
 * Unless a variant is fixed, the first inverse call for grid size N whose stream
 * is not being captured into a graph times every variant on its own work buffer
 * (the y pass before the window pass writes it, the other two on the first
 * catalogue) and keeps the fastest for the process and device; a call captured
 * before that uses variant 0.  Every variant computes the same transform (to
 * float32 rounding).
 *
 * hermes_fft_set_variant: fixes variant v (0 .. count - 1) for grid size N on the
 *   current device; v = -1 returns to autotuning (again on the next uncaptured call).
 * hermes_fft_variants: writes up to cap variants as {kind, E, W, minb} into desc
 *   (4 ints each) and the milliseconds of their timed trial into ms (-1 where not
 *   timed); *chosen = the tuned variant (-1 before tuning), *forced = the fixed
 *   one (-1 if none).  Any pointer may be NULL.  Returns the number of variants.
 * Errors: HERMES_ERR_ARG (N not one of 16 .. 1024, unknown pass, v out of range).
 */
#define HERMES_PASS_INV_Y 0
#define HERMES_PASS_WINDOW 1
#define HERMES_PASS_CONTRACT 2
#define HERMES_PASS_ZETA_Y 3
#define HERMES_PASS_ZETA_X 4
#define HERMES_PASS_ZETA_X_M0 5
int hermes_fft_set_variant(int N, int pass, int variant);
int hermes_fft_variants(int N, int pass, int *desc, double *ms, int cap, int *chosen, int *forced);

/* ------------------------------------------------------------------------
 * Device-memory accounting.
 *
 * hermes_device_bytes: bytes of device memory the context holds now (fields,
 * window tables, work and staging buffers, batched state); -1 for NULL.
 * hermes_estimate_bytes: what a context would hold after one request of the
 * given kind (stat as in hermes_request, n_bins shells, windows up to l_max,
 * n_points points, copied from host memory when host_inputs != 0); -1 on a
 * bad argument.  No device is needed.
 */
int64_t hermes_device_bytes(const hermes_ctx *ctx);
int64_t hermes_estimate_bytes(int N, int stat, int n_bins, int l_max, int64_t n_points, int host_inputs);

/* ------------------------------------------------------------------------
 * Request server: measurement requests of any grid size, catalogue size and
 * statistic, served with continuous batching on one GPU.
 *
 * Worker threads (n_streams, each with its own CUDA stream) take queued
 * requests as soon as a worker is free and the request's device footprint
 * (hermes_estimate_bytes) fits in hbm_budget next to the requests in flight
 * and the idle resident contexts; idle contexts are evicted least recently
 * used first.  A request passed over by 8 later ones blocks further
 * admissions until it fits.  Fields stay resident: a request whose field_id
 * (>= 0) names a field resident for the same L, N, p skips the scatter and the
 * forward transform and may pass pos = NULL, n = 0; requests for a field that
 * is being used wait for it.  Each result equals what the same calls on a
 * context of its own would give, to the rounding of float atomics.
 */
#define HERMES_STAT_XI 0
#define HERMES_STAT_XI_MULTIPOLES 1
#define HERMES_STAT_ZETA 2

typedef struct hermes_request {
    double L;                /* box side */
    int N, p;                /* grid (power of two, 16..1024) and B-spline order */
    int stat;                /* HERMES_STAT_* */
    const double *r_edges;   /* shells, as hermes_window_shells; copied at submit */
    int n_edges;
    const int *ells;         /* HERMES_STAT_XI_MULTIPOLES: orders; copied at submit */
    int n_ells;
    int l_max;               /* HERMES_STAT_ZETA: l_max */
    const float *pos;        /* as hermes_assign; must stay valid until the wait returns */
    const float *w;
    int64_t n;
    unsigned flags;
    int64_t field_id;        /* catalogue identity for reuse, or -1 */
    double *out;             /* result, caller-owned, written before the wait returns:
                                xi [n_bins]; xi_l [n_ells][n_bins]; zeta [l_max+1][n_bins][n_bins] */
} hermes_request;

typedef struct hermes_result {
    int status;              /* HERMES_OK or the error of the failing call */
    int reused_field;        /* 1 if a resident field served the request */
    double queue_ms;         /* submit -> start on a worker */
    double latency_ms;       /* submit -> result written */
    int64_t device_bytes;    /* the serving context's footprint afterwards */
    char msg[256];           /* error text */
} hermes_result;

typedef struct hermes_server hermes_server;

/* Errors: HERMES_ERR_ARG (bad device, n_streams outside 1..64, budget <= 0),
 * HERMES_ERR_CUDA (no GPU). */
int hermes_server_create(int device, int64_t hbm_budget, int n_streams, hermes_server **out);
/* Queues a request; *ticket identifies it.  Errors: HERMES_ERR_ARG (malformed
 * request), HERMES_ERR_STATE (server stopping).  Requests larger than the
 * whole budget complete with HERMES_ERR_NOMEM. */
int hermes_server_submit(hermes_server *srv, const hermes_request *req, int64_t *ticket);
/* Blocks until the request completes and returns its result (once per ticket).
 * Errors: HERMES_ERR_ARG (unknown ticket). */
int hermes_server_wait(hermes_server *srv, int64_t ticket, hermes_result *res);
/* stats[0..8] = completed, in flight, queued, bytes reserved, peak bytes
 * reserved, peak requests in flight, requests served from a resident field,
 * resident contexts, contexts evicted (the first n are written). */
int hermes_server_stats(hermes_server *srv, int64_t *stats, int n);
/* Fails queued requests with HERMES_ERR_STATE, lets running ones finish,
 * frees everything. */
int hermes_server_destroy(hermes_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* HERMES_H */
