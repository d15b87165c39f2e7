// Internal launcher declarations shared by the C ABI implementation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hermes {

constexpr int MAX_BATCH = 32;  // windows evaluated per launch of the first inverse pass (upper bound)

// Batched measurements: catalogues per call, and the per-catalogue strides of
// the field scalars (sum w, sum w^2, N^3/sum w, ...) and of the float self-pair tables.
constexpr int MAX_CATALOGUES = 1024;
constexpr int SCAL_STRIDE = 8;
constexpr int STAB_STRIDE = 512;

// Kernel classes reported by the tracer.
enum KernelId {
    K_SCATTER = 0, K_WEIGHT_SUMS, K_SELFPAIR, K_REDUCE, K_FINISH, K_FWD_Z_R2C, K_FWD_Y, K_FWD_X,
    K_INV_X_WINDOW, K_INV_Y, K_INV_Z_C2R_CONTRACT, K_ZETA_X, K_ZETA_Y, K_ZETA_Z_GRAM, K_NODES, K_INV_YZ_CONTRACT, K_ZETA_Z_GRAM_TC, K_KSPACE_HIST, K_KSPACE_CONTRACT, K_BATCH_GRAPH, K_SN_HIST, K_SN_CONTRACT, K_COMBINE, K_INV_Z_STORE, K_GATHER, K_WAIT_CHECK, K_DDD_FILTER, K_DDD_GRAM, K_COUNT
};

// Called around every kernel launch (phase 0 before, 1 after) on the launching stream.
struct Tracer {
    void* ctx;
    void (*mark)(void* ctx, int kernel_id, int phase, cudaStream_t st);
    void operator()(int id, int phase, cudaStream_t st) const {
        if (mark) mark(ctx, id, phase, st);
    }
};

// Radial tables are stored bin-fastest: rad[(l*Q + q)*nbp + b], nbp a multiple
// of 4, so one 16-byte load returns the values of 4 consecutive bins at |n|^2 = q.

// One batch of real (xi / xi_l) windows: consecutive bins b0 .. b0+S-1 of one
// even order l.  tab = rad + l*Q*nbp + b0; window s uses tab[q*nbp + s].
//
// Axisymmetric (cylindrical) windows, cyl = 1: K_{j,i}(n) = T_perp_i(n_x^2 + n_y^2)
// * T_par_j(|n_z|) * Phi^(n); tab is the transverse table indexed by q_perp =
// n_x^2 + n_y^2 (bin fastest), par = T_par_j over |n_z| in [0, N/2) for the
// batch's line-of-sight bin j; ell and scale are unused.
// Ring windows (par_stride > 0): window s of the batch has its own line-of-sight
// row, par + s * par_stride, paired with transverse column s (a list of (R, H)
// rings instead of a product grid of bins).
struct WinBatch {
    const float* tab;
    int nbp;
    int S;
    int ell;
    float scale;  // (2l+1) i^l, real for even l
    int cyl = 0;
    const float* par = nullptr;
    int par_stride = 0;
};

// One batch of complex harmonic windows: all bins of a fixed (l, m).
// tab = rad + l*Q*nbp; bin b uses tab[q*nbp + b].
// pack = 1 (m = 0, whose fields are real): bins 2f and 2f+1 share complex field f as
// its real and imaginary parts, so (S + 1) / 2 fields are transformed instead of S.
// tab2 != nullptr: bins 8..S-1 of the batch come from tab2 (bin b uses tab2[q*nbp + b - 8]),
// so one launch can pair two blocks of 8 bins that are not adjacent in the table.
struct HarmBatch {
    const float* tab;
    const float* tab2 = nullptr;
    int nbp;
    int S;      // number of bins (<= 16)
    int ell, m;
    float ylm_norm;  // N_lm (-1)^m (2m-1)!!  times 4 pi
    int pack = 0;
};

// Orders of one k-space evaluation (even l, at most 8).  cyl = 1: the entries
// are line-of-sight bins j of an axisymmetric window instead, each weighting a
// mode by par[j*(N/2) + |n_z|], the histogram is indexed by q_perp = n_x^2 + n_y^2
// and the contraction constant is 1.
// diag = 1 (ring windows): entry o is window ell[o], whose line-of-sight row and
// transverse column are both ell[o]; the contraction yields one value per entry.
struct KsOrders {
    int n;
    int ell[8];
    int cyl = 0;
    const float* par = nullptr;
    int diag = 0;
};

struct Tables {
    const float2* tw;     // twiddle tables, layout in fft_core.cuh
    const float* phi;     // [N]  sinc^{2p}(pi n / N), FFT order
    const float* stab;    // [p^3] self-pair table (float); batched: catalogue c at stab + c*STAB_STRIDE
};

// scatter.cu
cudaError_t launch_scatter(int N, int p, const float* pos, const float* w, int64_t n, float* grid, float s,
                           int wrap, unsigned* err, cudaStream_t st, const Tracer& tr);
// Shared-memory-privatised scatter into grid (no clearing needed; no global
// atomics on the grid).  Scratch: tile_of, perm [n] ints; counts, cursor
// [ntiles] ints, offs [ntiles + 1] ints; regions [scatter_tiled_region_floats] floats.
size_t scatter_tiled_region_floats(int N, int p);
int scatter_tiled_tiles(int N);
cudaError_t launch_scatter_tiled(int N, int p, const float* pos, const float* w, int64_t n, float* grid, float s,
                                 int wrap, unsigned* err, int* tile_of, int* perm, int* counts, int* offs,
                                 int* cursor, float* regions, cudaStream_t st, const Tracer& tr);
// catalogues c0 .. c1-1; catalogue c: points [offs[c], offs[c+1]) (device
// offsets), grid + c*N^3; n_max bounds the points of the group (sizes the grid)
cudaError_t launch_scatter_batch(int N, int p, const float* pos, const float* w, const int64_t* offs, int c0, int c1,
                                 int64_t n_max, float* grid, float s, int wrap, unsigned* err, cudaStream_t st,
                                 const Tracer& tr);
cudaError_t launch_nodes(int N, int p, const float* pos, int64_t n, float s, int wrap, int* first, float* wts,
                         unsigned* err, cudaStream_t st, const Tracer& tr);
// offs != nullptr: per-catalogue partials, [ncat][2][nblk] (sums) and [ncat][p^3][nblk] (self-pair)
cudaError_t launch_weight_sums(const float* w, int64_t n, double* part, int nblk, cudaStream_t st, const Tracer& tr,
                               const int64_t* offs = nullptr, int ncat = 1);
cudaError_t launch_selfpair(int N, int p, const float* pos, const float* w, int64_t n, float s, double* part,
                            int nblk, cudaStream_t st, const Tracer& tr, const int64_t* offs = nullptr,
                            int ncat = 1);
cudaError_t launch_reduce_rows(const double* part, int rows, int cols, double* out, cudaStream_t st, const Tracer& tr);
cudaError_t launch_reduce_rows_strided(const double* part, int rows, int cols, int S, double* out, int out_stride,
                                       cudaStream_t st, const Tracer& tr);
cudaError_t launch_finish_field(const double* sums, const double* stab_d, int p3, float* stab_f, int N,
                                double* scal, cudaStream_t st, const Tracer& tr);
cudaError_t launch_finish_batch(const double* sums, const double* sp, int p3, float* stab_f, int N, double* scal,
                                int ncat, cudaStream_t st, const Tracer& tr);
cudaError_t launch_xi_batch_finish(const double* dd, const double* sn, const double* scal, int ncat, int nwin, int N,
                                   double* out, cudaStream_t st, const Tracer& tr);

// fft_passes.cu.  ncat > 1: catalogue c uses grid + c*N^3, spec + c*N*N*(N/2),
// scal + c*SCAL_STRIDE; the inverse work buffer is [ncat][S][N][N][N/2] and the
// partials are [ncat][S][blocks].
cudaError_t launch_forward(int N, float* grid, float2* spec, const double* scal, const Tables& tb,
                           cudaStream_t st, const Tracer& tr, int ncat = 1);
int inv_x_blocks(int N);
// Variants of the tuned FFT passes and their autotuner; -1 on a bad argument.
int fft_variants(int N, int pass, int* desc, double* ms, int cap, int* chosen, int* forced);
int fft_set_variant(int N, int pass, int variant);
// The zeta_l y pass (pass 3): the variant for nf fields of N^3 (tuned on the first of
// them, in place, when untuned and not capturing: call before the x pass writes them),
// and its launch.
int zeta_y_variant(int N, float2* fields, int nf, const float2* tw, cudaStream_t st);
// The tuned variant of (N, pass): the fixed or tuned one, else (timing trial(v, arg), one
// launch of variant v, for every variant when st is not capturing) the fastest; 0 while
// capturing before any tuning.
int tuned_variant(int N, int pass, cudaStream_t st, cudaError_t (*trial)(int v, void* arg), void* arg);
// paired: the fields are in the paired order of the zeta_l x pass's paired variant, which
// only the variants for which zeta_y_reads_paired holds can read.
cudaError_t launch_zeta_y(int N, int var, float2* fields, int nf, const float2* tw, cudaStream_t st,
                          bool paired = false);
bool zeta_y_reads_paired(int N, int var);
int inv_z_blocks(int N);        // blocks of the last inverse pass for one catalogue (fused y-z if enabled)
int inv_z_blocks_plain(int N);  // the same for the three-pass form (always used when ncat > 1)
// window multiply + inverse transforms + cell contraction of one window batch;
// dd_part: [ncat][S][blocks] partial sums of delta * filtered field
cudaError_t launch_inverse_xi(int N, const float2* spec, float2* work, const float* delta, const WinBatch& wb,
                              const Tables& tb, double* dd_part, unsigned* err, cudaStream_t st, const Tracer& tr,
                              int ncat = 1);
// delta~ = iFT(spec * K) / N^3 written to out (N^3 floats) for one window (wb.S = 1);
// work holds one half spectrum
cudaError_t launch_smooth_field(int N, const float2* spec, float2* work, float* out, const WinBatch& wb,
                                const Tables& tb, cudaStream_t st, const Tracer& tr);
// forward transform of a field as it is (no eps -> delta conversion); keep_dc = 1
// keeps the k = 0 mode (otherwise it is set to 0)
cudaError_t launch_delta_to_spec(int N, float* grid, float2* spec, const double* scal, const Tables& tb,
                                 cudaStream_t st, const Tracer& tr, int keep_dc = 0);
// Smoothed density at points: rho_i = 1 + sum_l phi_l(x_i) field_l (the scatter's node
// rule and weights), then the mark: kind 0 rho; 1 (max(rho - self, 0) + b)^a;
// 2 ((b + 1) / (b + max(rho - self, 0)))^a.  err bit 1 marks a rejected coordinate.
cudaError_t launch_gather_marks(int N, int p, const float* pos, int64_t n, const float* field, float s, int wrap,
                                int kind, float a, float b, float self, float* out, unsigned* err, cudaStream_t st,
                                const Tracer& tr);
// Landy-Szalay difference field: grid <- (grid - alpha * rgrid) * inv_ebar (n cells), and the
// combined float self-pair table stab_f[e] = stab_d[e] + alpha^2 rstab_d[e] (p3 entries)
cudaError_t launch_combine_randoms(float* grid, const float* rgrid, size_t n, float alpha, float inv_ebar,
                                   const double* stab_d, const double* rstab_d, double alpha2, float* stab_f, int p3,
                                   cudaStream_t st, const Tracer& tr);

// kspace.cu
// self_only = 0: A_l(q) of the Parseval route; self_only = 1: the self-pair
// histogram B_l(q) = sum_{|n|^2=q} w_z Phi^ L_l S^ alone (spec and scal unused)
cudaError_t launch_kspace_hist(int N, const float2* spec, const Tables& tb, int P, const double* scal,
                               const KsOrders& ko, double* hist, int64_t Q, cudaStream_t st, const Tracer& tr,
                               int self_only = 0);
// out[o*nb + b] = c_l sum_q T_{b,l}(q) hist[o*Q + q] / N^6, c_l = (2l+1) i^l;
// ko.diag: out[o] = sum_q T_{ell[o]}(q) hist[o*Q + q] / N^6 (one column per entry)
cudaError_t launch_kspace_contract(const float* rad, int nbp, int64_t Q, const KsOrders& ko, const double* hist,
                                   int N, double* out, int nb, cudaStream_t st, const Tracer& tr,
                                   int trace_id = K_KSPACE_CONTRACT);

// wait_check.cu: one thread waits, with the bounded mbarrier wait of the bulk-copy
// pipelines, on a barrier phase that nothing completes; err bit 4 marks the expiry
cudaError_t launch_wait_unarrived(unsigned* err, cudaStream_t st, const Tracer& tr);

// fft_passes.cu: the real filtered fields iFT(spec * K_s) / N^3 of a window batch
// (wb.S <= 16 windows, tab 16-byte aligned) into out + s * N^3; work holds S half spectra
cudaError_t launch_filtered_fields(int N, const float2* spec, float2* work, float* out, const WinBatch& wb,
                                   const Tables& tb, cudaStream_t st, const Tracer& tr);

// ddd.cu: the 3PCF monopole by triple connection coefficients, as an exact Gauss-Legendre
// quadrature of the triple product of spline fields (n_g = ddd_samples(p) samples per axis
// and knot cell; the sample t_g of cell c reads taps c + j0 + j, j < p, with weights b[g][j]).
__host__ __device__ constexpr int ddd_samples(int p) { return (3 * p - 1) / 2; }
constexpr int DDD_MAX_SAMPLES = 11;  // p = 8
struct DddYZ {
    float by[8], bz[8];  // the y and z taps of one (g_y, g_z) sample pair
    int j0;
};
struct DddTaps {
    float bx[DDD_MAX_SAMPLES][8];  // the x taps of every g_x
    float wx[DDD_MAX_SAMPLES];     // the x Gauss weights
    double wyz;                    // w_gy * w_gz
    int j0;
    // the Gram's 17 field slots: slot 0 delta, slots 1..8 the row block's bins, 9..16 the
    // column block's; fld[slot] = the field's index in Y, -1 for an empty slot
    int fld[17];
    int tile0;  // one warp per block: its tile, 0 = (rows, rows) upper triangle, 1 = (rows, columns)
};
// Y_f = the y and z filters of nf fields of N^3 (in and out [nf][N][N][N])
cudaError_t launch_ddd_filter_yz(int N, int p, const float* in, float* out, int nf, const DddYZ& tp,
                                 cudaStream_t st, const Tracer& tr);
// the x filters and the weighted Gram of the fields tp.fld of Y (N >= 16), added into part
// [ddd_gram_blocks(N, nw)][3][64], times wyz.  nw = 3: tiles {(rows, rows), (rows, columns),
// (columns, columns)} in tiles 0, 1, 2; nw = 1: tile tp.tile0 alone, in tile 0.  Entry 8 a + b
// of a tile = slots (row a, column b); the diagonal tiles keep the upper triangle.
int ddd_gram_blocks(int N, int nw);
cudaError_t launch_ddd_gram(int N, int p, const float* Y, int nw, const DddTaps& tp, double* part, cudaStream_t st,
                            const Tracer& tr);

// zeta.cu
int zeta_z_blocks(int N);
cudaError_t launch_zeta_lm(int N, const float2* spec, float2* fields, const float* delta, const HarmBatch& hb,
                           const Tables& tb, double* gram_part, unsigned* err, cudaStream_t st, const Tracer& tr);

}  // namespace hermes
