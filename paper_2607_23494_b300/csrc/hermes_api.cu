// C ABI of the field-window estimator: context, input validation, float64
// window tables and orchestration of the kernels.  See include/hermes.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hermes.h"
#include "kernels.h"
#include "common.cuh"
#include "fft_core.cuh"

using namespace hermes;

struct BatchState;  // batched measurements (defined with hermes_xi_multipoles_batch)
void batch_free(BatchState* b);

struct hermes_ctx {
    double L = 0;
    int N = 0, p = 0, j = 0, H = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    // device buffers
    float* grid = nullptr;       // N^3: eps, then delta
    float2* spec = nullptr;      // N*N*H half spectrum
    float2* work = nullptr;      // batch of filtered spectra
    size_t work_bytes = 0;
    float2* zfields = nullptr;   // harmonic fields (full complex)
    size_t zfields_bytes = 0;
    double* part = nullptr;      // block partial sums
    size_t part_cap = 0;         // doubles
    double* red = nullptr;       // reduced results
    size_t red_cap = 0;          // doubles
    double* scal = nullptr;      // [0] sum w [1] sum w^2 [2] N^3/sum w [3..] reduced sums
    double* stab_d = nullptr;    // p^3
    float* stab_f = nullptr;     // p^3
    unsigned* err = nullptr;
    float2* tw = nullptr;
    float* phi = nullptr;
    float* stage_pos = nullptr;
    float* stage_w = nullptr;
    size_t stage_cap = 0;        // points
    double* host_buf = nullptr;  // pinned readback
    size_t host_cap = 0;
    // bins
    int n_bins = 0, l_max = -1;
    int64_t Q = 0;
    int nbp = 0;                 // bins padded to a multiple of 4
    std::vector<double> edges;
    float* rad = nullptr;        // [(l*Q + q)*nbp + b]
    // axisymmetric windows: transverse table [q_perp*cyl_nbp + i], line-of-sight [j*H + |n_z|]
    float* cyl_perp = nullptr;
    float* cyl_par = nullptr;
    int cyl_nperp = 0, cyl_npar = 0, cyl_nbp = 0;
    int64_t cyl_Q = 0;
    // ring windows (hermes_window_rings): window w pairs transverse column w with
    // line-of-sight row w instead of spanning the product grid
    bool cyl_ring = false;
    // explicit random catalogue (Landy-Szalay): raw field, its transform (k = 0 kept),
    // self-pair table; rscal[2] = 1 so the histogram kernel subtracts S^ unscaled
    float* rgrid = nullptr;
    float2* rspec = nullptr;
    double* rstab_d = nullptr;
    float* rstab_f = nullptr;
    double* rscal = nullptr;
    double sum_wr = 0;
    bool have_randoms = false;
    float* smooth_tab = nullptr;  // one-bin smoothing table [q*4] (density marks)
    // tiled scatter scratch: per-point tile and permutation, per-tile counts / offsets /
    // cursors, and the per-tile deposit regions
    int* ts_tile_of = nullptr;
    int* ts_perm = nullptr;
    size_t ts_pts_cap = 0;
    int* ts_tiles = nullptr;      // [counts | offs (+1) | cursor]
    float* ts_regions = nullptr;
    size_t ts_regions_cap = 0;    // floats
    // state
    bool have_field = false;
    double sum_w = 0, sum_w2 = 0;
    std::string msg;
    // tracing: launch counter always on; event pairs per launch when enabled
    int64_t launches = 0;
    bool trace_on = false;
    struct Pending {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open_ev = nullptr;
    double trace_ms[K_COUNT] = {0};
    int64_t trace_n[K_COUNT] = {0};
    Tracer tracer{nullptr, nullptr};
    BatchState* batch = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(hermes_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->msg = buf;
    }
    return code;
}

int cuda_fail(hermes_ctx* c, cudaError_t e, const char* what) {
    cudaGetLastError();  // clear sticky non-fatal errors
    if (e == cudaErrorMemoryAllocation) return fail(c, HERMES_ERR_NOMEM, "%s: out of device memory", what);
    return fail(c, HERMES_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return cuda_fail(c, _e, what);   \
    } while (0)

// Every device allocation of the library goes through here.  The test hook
// hermes_debug_fail_allocs makes the next few report out of memory without
// allocating, so the error paths can be exercised without exhausting a GPU.
//
// Context memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// context's stream, named by AllocStream for the duration of each entry point):
// a context that grows or releases a buffer then never waits for the whole
// device, so contexts on other streams (the request server's workers) keep
// running.  Every entry point synchronises its stream before returning, so a
// buffer is idle whenever it is freed or the context's stream is changed.
std::atomic<int> g_fail_allocs{0};
thread_local cudaStream_t t_alloc_stream = nullptr;

struct AllocStream {
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
    ~AllocStream() { t_alloc_stream = prev; }
};

// The device's default pool keeps up to 8 GiB of freed memory between synchronisations
// (released beyond that), so buffers that are freed and grown again are cheap.
void pool_setup(int dev) {
    static std::mutex mu;
    static bool done[256] = {false};
    if (dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = (uint64_t)8 << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
            *ptr = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    if (t_alloc_stream) return cudaMallocAsync(ptr, bytes, t_alloc_stream);
    return cudaMalloc(ptr, bytes);
}

void dev_free(void* ptr) {
    if (!ptr) return;
    if (t_alloc_stream) cudaFreeAsync(ptr, t_alloc_stream);
    else cudaFree(ptr);
}

// Host-to-device upload into a context buffer, ordered after its allocation on stream st;
// returns once the host source may be reused.
cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    return e != cudaSuccess ? e : cudaStreamSynchronize(st);
}

template <class T>
cudaError_t grow(T*& ptr, size_t& cap_bytes, size_t need_bytes) {
    if (need_bytes <= cap_bytes && ptr) return cudaSuccess;
    if (ptr) dev_free(ptr);
    ptr = nullptr;
    cap_bytes = 0;
    cudaError_t e = dev_malloc((void**)&ptr, need_bytes);
    if (e == cudaSuccess) cap_bytes = need_bytes;
    return e;
}

cudaError_t grow_doubles(double*& ptr, size_t& cap, size_t need) {
    size_t bytes = cap * sizeof(double);
    cudaError_t e = grow(ptr, bytes, need * sizeof(double));
    cap = bytes / sizeof(double);
    return e;
}

// ---------------------------------------------------------------------------
// float64 window mathematics (host)
//
// I_l(x) = int_0^x t^2 j_l(t) dt gives the r^2-weighted bin average
//   <j_l>_b(k) = 3 [I_l(k r_hi) - I_l(k r_lo)] / (k^3 (r_hi^3 - r_lo^3)).
// Small x: the power series of j_l integrated term by term.  Larger x: the
// closed forms built from the sine integral with the recurrences
//   H_0 = Si, H_1 = 1 - j_0, (m+1) H_{m+1} = m H_{m-1} - (2m+1) j_m       (H_m = int j_m)
//   J_0 = 1 - cos, J_1 = Si - sin, J_m = (2m-1) H_{m-1} - J_{m-2}        (J_m = int t j_m)
//   I_0 = sin - x cos, I_1 = 2 - 2 cos - x sin, I_l = (2l-1) J_{l-1} - I_{l-2}
// which follow from j_l = (2l-1)/t j_{l-1} - j_{l-2} and
// (2m+1) j_m' = m j_{m-1} - (m+1) j_{m+1}.

// Sine integral Si(x), x >= 0: power series for x <= 2, otherwise
// Si = pi/2 + Im E1(ix) with E1 evaluated by its continued fraction
// E1(z) = e^{-z} / (z + 1 - 1^2/(z + 3 - 2^2/(z + 5 - ...))) (modified Lentz).
double sine_integral(double x) {
    if (x <= 2.0) {
        double sum = 0.0, term = x;  // term = (-1)^k x^{2k+1} / (2k+1)!
        for (int k = 0; k < 40; ++k) {
            const double add = term / (2.0 * k + 1.0);
            sum += add;
            if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
            term *= -x * x / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
        return sum;
    }
    typedef std::complex<double> cd;
    const double tiny = 1e-300;
    cd b(1.0, x);
    cd cc = 1.0 / tiny;
    cd d = 1.0 / b;
    cd h = d;
    for (int i = 1; i < 100000; ++i) {
        const double a = -(double)i * (double)i;
        b += 2.0;
        d = 1.0 / (a * d + b);
        cc = b + a / cc;
        const cd del = cc * d;
        h *= del;
        if (std::fabs(del.real() - 1.0) + std::fabs(del.imag()) < 1e-16) break;
    }
    h *= cd(std::cos(x), -std::sin(x));
    return 1.5707963267948966192 + h.imag();
}

double dfact2(int n) {  // n!! for odd n >= -1
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

// I_l(x) for l = 0..lmax into out[l].
void bessel_moment_all(double x, int lmax, double* out) {
    if (x == 0.0) {
        for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
        return;
    }
    const double xs = x * x;
    // series where it is accurate: x < l + 4
    int first_rec = lmax + 1;
    for (int l = 0; l <= lmax; ++l) {
        if (x < l + 4.0) {
            double s = 1.0, sum = 1.0 / (l + 3.0);
            for (int k = 1; k < 200; ++k) {
                s *= -0.5 * xs / ((double)k * (2.0 * l + 2.0 * k + 1.0));
                const double add = s / (2.0 * k + l + 3.0);
                sum += add;
                if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
            }
            out[l] = sum * std::pow(x, l + 3) / dfact2(2 * l + 1);
        } else if (first_rec > lmax) {
            first_rec = l;
        }
    }
    if (first_rec > lmax) return;
    // closed forms for l >= first_rec (used for the orders with x >= l + 4)
    const double sn = std::sin(x), cs = std::cos(x), si = sine_integral(x);
    const int M = lmax + 1;
    std::vector<double> jl(M + 1), Hm(M + 1), Jm(M + 1), Il(M + 1);
    jl[0] = sn / x;
    if (M >= 1) jl[1] = sn / xs - cs / x;
    for (int m = 1; m < M; ++m) jl[m + 1] = (2.0 * m + 1.0) / x * jl[m] - jl[m - 1];
    Hm[0] = si;
    Hm[1] = 1.0 - jl[0];
    for (int m = 1; m + 1 <= M; ++m) Hm[m + 1] = (m * Hm[m - 1] - (2.0 * m + 1.0) * jl[m]) / (m + 1.0);
    Jm[0] = 1.0 - cs;
    Jm[1] = si - sn;
    for (int m = 2; m <= M; ++m) Jm[m] = (2.0 * m - 1.0) * Hm[m - 1] - Jm[m - 2];
    Il[0] = sn - x * cs;
    Il[1] = 2.0 - 2.0 * cs - x * sn;
    for (int l = 2; l <= lmax; ++l) Il[l] = (2.0 * l - 1.0) * Jm[l - 1] - Il[l - 2];
    // only where x >= l + 4: below that the recurrence cancels and the series (above) holds
    for (int l = first_rec; l <= lmax; ++l)
        if (!(x < l + 4.0)) out[l] = Il[l];
}

// out[((b*(lmax+1)) + l)*Q + q] = <j_l>_b(k_q), k_q = 2 pi sqrt(q) / L.
void build_shell_tables(double L, int64_t Q, const double* edges, int n_edges, int lmax, double* out) {
    const int nb = n_edges - 1;
    const int LM = lmax + 1;
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        std::vector<double> Ie((size_t)n_edges * LM);
        const int64_t chunk = 256;
        for (;;) {
            const int64_t q0 = next.fetch_add(chunk);
            if (q0 >= Q) break;
            const int64_t q1 = std::min(Q, q0 + chunk);
            for (int64_t q = q0; q < q1; ++q) {
                if (q == 0) {
                    for (int b = 0; b < nb; ++b)
                        for (int l = 0; l < LM; ++l) out[((size_t)b * LM + l) * Q] = (l == 0) ? 1.0 : 0.0;
                    continue;
                }
                const double k = 2.0 * M_PI * std::sqrt((double)q) / L;
                for (int e = 0; e < n_edges; ++e) bessel_moment_all(k * edges[e], lmax, &Ie[(size_t)e * LM]);
                const double k3 = k * k * k;
                for (int b = 0; b < nb; ++b) {
                    const double lo = edges[b], hi = edges[b + 1];
                    const double den = k3 * (hi * hi * hi - lo * lo * lo) / 3.0;
                    for (int l = 0; l < LM; ++l)
                        out[((size_t)b * LM + l) * Q + q] =
                            (Ie[(size_t)(b + 1) * LM + l] - Ie[(size_t)b * LM + l]) / den;
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (unsigned i = 1; i < nth; ++i) th.emplace_back(worker);
    worker();
    for (auto& t : th) t.join();
}

int64_t table_len(int N) {
    const int64_t h = N / 2 - 1;
    return 3 * h * h + 1;
}

bool valid_N(int N) { return N >= 16 && N <= 1024 && (N & (N - 1)) == 0; }

// Windows per launch of the inverse passes: up to 16 within an 8 GiB work
// buffer, a multiple of 4 (bin offsets b0 = 0, S, 2S, ... must stay 16-byte
// aligned in the tables), at least 4, and one batch per order when the bins fit.
size_t xi_window_S(int N, int nb) {
    const size_t win_bytes = (size_t)N * N * (N / 2) * sizeof(float2);
    int S = (int)std::min<size_t>(16, ((size_t)8 << 30) / win_bytes) & ~3;
    S = std::max(S, 4);
    return (size_t)std::min(S, std::max(nb, 1));
}

Tables tables_of(const hermes_ctx* c) {
    Tables t;
    t.tw = c->tw;
    t.phi = c->phi;
    t.stab = c->stab_f;
    return t;
}

cudaEvent_t pool_event(hermes_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void trace_mark(void* vc, int id, int phase, cudaStream_t st) {
    hermes_ctx* c = (hermes_ctx*)vc;
    if (phase == 0) ++c->launches;
    if (!c->trace_on) return;
    if (phase == 0) {
        c->open_ev = pool_event(c);
        if (c->open_ev) cudaEventRecord(c->open_ev, st);
    } else if (c->open_ev) {
        cudaEvent_t b = pool_event(c);
        if (b) {
            cudaEventRecord(b, st);
            c->pending.push_back({id, c->open_ev, b});
        } else {
            c->pool.push_back(c->open_ev);
        }
        c->open_ev = nullptr;
    }
}

// Fold finished event pairs into the per-kernel totals (synchronises the stream).
void trace_collect(hermes_ctx* c) {
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            c->trace_ms[p.id] += ms;
            c->trace_n[p.id] += 1;
        }
        c->pool.push_back(p.a);
        c->pool.push_back(p.b);
    }
    cudaGetLastError();
    c->pending.clear();
}

int ensure_host(hermes_ctx* c, size_t n) {
    if (n <= c->host_cap) return HERMES_OK;
    if (c->host_buf) cudaFreeHost(c->host_buf);
    c->host_buf = nullptr;
    c->host_cap = 0;
    if (cudaMallocHost((void**)&c->host_buf, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HERMES_ERR_NOMEM, "pinned host buffer of %zu doubles", n);
    }
    c->host_cap = n;
    return HERMES_OK;
}

// Grows the tiled-scatter scratch for n points (tile tables and regions are sized once).
cudaError_t tiled_scratch(hermes_ctx* c, int64_t n) {
    cudaError_t e;
    if ((size_t)n > c->ts_pts_cap) {
        dev_free(c->ts_tile_of);
        dev_free(c->ts_perm);
        c->ts_tile_of = nullptr;
        c->ts_perm = nullptr;
        c->ts_pts_cap = 0;
        if ((e = dev_malloc((void**)&c->ts_tile_of, (size_t)n * sizeof(int))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&c->ts_perm, (size_t)n * sizeof(int))) != cudaSuccess) return e;
        c->ts_pts_cap = (size_t)n;
    }
    if (!c->ts_tiles) {
        const size_t nt = (size_t)scatter_tiled_tiles(c->N);
        if ((e = dev_malloc((void**)&c->ts_tiles, (3 * nt + 1) * sizeof(int))) != cudaSuccess) return e;
    }
    const size_t rf = scatter_tiled_region_floats(c->N, c->p);
    if (rf > c->ts_regions_cap) {
        dev_free(c->ts_regions);
        c->ts_regions = nullptr;
        c->ts_regions_cap = 0;
        if ((e = dev_malloc((void**)&c->ts_regions, rf * sizeof(float))) != cudaSuccess) return e;
        c->ts_regions_cap = rf;
    }
    return cudaSuccess;
}

// The tiled scatter has a fixed cost that grows with N^3 (it writes and re-reads one
// (16+p-1)^3 region per 16^3 tile); per-point global atomics on a cleared grid cost more per
// point but little per cell.  Measured on B300 (p = 4, whole hermes_assign): the atomics are
// faster below about 1.2e6 points at 512^3 and 4e6 at 256^3, and at every size up to 1e7 at
// 128^3; 1024^3 (eight times the fixed cost of 512^3) is extrapolated to 9e6.
// HERMES_SCATTER=tiled or =atomic forces one form (tests run both on every order p).
bool sparse_scatter(int N, int64_t n) {
    const char* force = getenv("HERMES_SCATTER");
    if (force && std::strcmp(force, "tiled") == 0) return false;
    if (force && std::strcmp(force, "atomic") == 0) return true;
    if (N <= 128) return true;
    const double limit = N == 256 ? 4e6 : (N == 512 ? 1.2e6 : 9e6);
    return (double)n < limit;
}

// Scatter of n points into dst (an N^3 grid): the shared-memory tiled form for dense
// catalogues (no clearing needed), global atomics on a cleared grid for sparse ones.
cudaError_t scatter_tiled(hermes_ctx* c, const float* pos, const float* w, int64_t n, float* dst, float s, int wrap,
                          cudaStream_t st) {
    if (sparse_scatter(c->N, n)) {
        cudaError_t e = cudaMemsetAsync(dst, 0, (size_t)c->N * c->N * c->N * sizeof(float), st);
        if (e != cudaSuccess) return e;
        return launch_scatter(c->N, c->p, pos, w, n, dst, s, wrap, c->err, st, c->tracer);
    }
    cudaError_t e = tiled_scratch(c, n);
    if (e != cudaSuccess) return e;
    const size_t nt = (size_t)scatter_tiled_tiles(c->N);
    int* counts = c->ts_tiles;
    int* offs = counts + nt;
    int* cursor = offs + nt + 1;
    return launch_scatter_tiled(c->N, c->p, pos, w, n, dst, s, wrap, c->err, c->ts_tile_of, c->ts_perm, counts, offs,
                                cursor, c->ts_regions, st, c->tracer);
}

int check_ctx(hermes_ctx* c) {
    if (!c) return HERMES_ERR_ARG;
    c->msg.clear();
    return HERMES_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int hermes_create(double L, int N, int p, int j, hermes_ctx** out) {
    if (!out) return HERMES_ERR_ARG;
    *out = nullptr;
    if (!(L > 0.0) || !std::isfinite(L)) return HERMES_ERR_ARG;
    if (j < 4 || j > 10 || N != (1 << j) || !valid_N(N)) return HERMES_ERR_ARG;
    if (p < 1 || p > 8 || 2 * p - 1 > N) return HERMES_ERR_ARG;
    hermes_ctx* c = new (std::nothrow) hermes_ctx;
    if (!c) return HERMES_ERR_NOMEM;
    c->L = L;
    c->N = N;
    c->p = p;
    c->j = j;
    c->H = N / 2;
    c->tracer.ctx = c;
    c->tracer.mark = trace_mark;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return HERMES_ERR_CUDA;
    }
    DeviceGuard g(c->device);
    auto bail = [&](int code) {
        hermes_destroy(c);
        return code;
    };
    const size_t n3 = (size_t)N * N * N;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(HERMES_ERR_CUDA);
    c->stream = c->own_stream;
    pool_setup(c->device);
    AllocStream as_(c->own_stream);  // every buffer of the context comes from the stream-ordered pool
    if (dev_malloc((void**)&c->grid, n3 * sizeof(float)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->spec, (size_t)N * N * c->H * sizeof(float2)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->scal, 8 * sizeof(double)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->stab_d, 512 * sizeof(double)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->stab_f, 512 * sizeof(float)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->err, sizeof(unsigned)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->tw, TW_ENTRIES * sizeof(float2)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    if (dev_malloc((void**)&c->phi, N * sizeof(float)) != cudaSuccess) return bail(HERMES_ERR_NOMEM);
    // the allocations are ordered on the context's stream: complete them before the copies
    // below (legacy stream) and before any other stream uses the buffers
    if (cudaStreamSynchronize(c->own_stream) != cudaSuccess) return bail(HERMES_ERR_CUDA);
    // multi-level twiddles tw[L + j] = e^{-2 pi i j / L} (L = 2, 4, ..., TW) and
    // Phi^(n) = sinc^{2p}(pi n / N), in float64, stored as float32
    std::vector<float2> tw(TW_ENTRIES, make_float2(0.f, 0.f));
    for (int Lv = 2; Lv <= TW; Lv *= 2)
        for (int i = 0; i < Lv; ++i) {
            const double a = -2.0 * M_PI * (double)i / (double)Lv;
            tw[Lv + i] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    // radix-8 stage twiddles e^{-2 pi i k r / (8 NS)}, [r-1][k] per NS
    for (int NS = 2; 8 * NS <= TW; NS *= 2)
        for (int r = 1; r < 8; ++r)
            for (int k = 0; k < NS; ++k) {
                const double a = -2.0 * M_PI * (double)k * (double)r / (8.0 * NS);
                tw[STAGE_TW + 7 * (NS - 1) + (r - 1) * NS + k] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
    std::vector<float> ph(N);
    for (int k = 0; k < N; ++k) {
        const int n = k < N / 2 ? k : k - N;
        const double x = M_PI * (double)n / (double)N;
        const double s = (n == 0) ? 1.0 : std::sin(x) / x;
        ph[k] = (float)std::pow(s, 2 * p);
    }
    if (cudaMemcpy(c->tw, tw.data(), TW_ENTRIES * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) return bail(HERMES_ERR_CUDA);
    if (cudaMemcpy(c->phi, ph.data(), N * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return bail(HERMES_ERR_CUDA);
    if (cudaMemset(c->stab_f, 0, 512 * sizeof(float)) != cudaSuccess) return bail(HERMES_ERR_CUDA);
    if (ensure_host(c, 1024) != HERMES_OK) return bail(HERMES_ERR_NOMEM);
    *out = c;
    return HERMES_OK;
}

int hermes_destroy(hermes_ctx* c) {
    if (!c) return HERMES_OK;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    dev_free(c->grid);
    dev_free(c->spec);
    dev_free(c->work);
    dev_free(c->zfields);
    dev_free(c->part);
    dev_free(c->red);
    dev_free(c->scal);
    dev_free(c->stab_d);
    dev_free(c->stab_f);
    dev_free(c->err);
    dev_free(c->tw);
    dev_free(c->phi);
    dev_free(c->stage_pos);
    dev_free(c->stage_w);
    dev_free(c->rad);
    dev_free(c->cyl_perp);
    dev_free(c->cyl_par);
    dev_free(c->rgrid);
    dev_free(c->rspec);
    dev_free(c->rstab_d);
    dev_free(c->rstab_f);
    dev_free(c->rscal);
    dev_free(c->smooth_tab);
    dev_free(c->ts_tile_of);
    dev_free(c->ts_perm);
    dev_free(c->ts_tiles);
    dev_free(c->ts_regions);
    batch_free(c->batch);
    c->batch = nullptr;
    if (c->host_buf) cudaFreeHost(c->host_buf);
    for (auto& p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    cudaGetLastError();
    delete c;
    return HERMES_OK;
}

int hermes_fft_set_variant(int N, int pass, int variant) {
    return fft_set_variant(N, pass, variant) == 0 ? HERMES_OK : HERMES_ERR_ARG;
}

int hermes_fft_variants(int N, int pass, int* desc, double* ms, int cap, int* chosen, int* forced) {
    const int n = fft_variants(N, pass, desc, ms, std::max(cap, 0), chosen, forced);
    return n < 0 ? HERMES_ERR_ARG : n;
}

int hermes_release_buffers(hermes_ctx* c) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    CK(cudaStreamSynchronize(c->stream), "release buffers");
    dev_free(c->work);
    dev_free(c->zfields);
    dev_free(c->stage_pos);
    dev_free(c->stage_w);
    dev_free(c->ts_tile_of);
    dev_free(c->ts_perm);
    dev_free(c->ts_regions);
    c->work = nullptr;
    c->zfields = nullptr;
    c->stage_pos = c->stage_w = nullptr;
    c->ts_tile_of = c->ts_perm = nullptr;
    c->ts_regions = nullptr;
    c->work_bytes = c->zfields_bytes = 0;
    c->stage_cap = c->ts_pts_cap = c->ts_regions_cap = 0;
    return HERMES_OK;
}

int hermes_set_stream(hermes_ctx* c, void* s) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    c->stream = s ? (cudaStream_t)s : c->own_stream;
    return HERMES_OK;
}

const char* hermes_last_error(const hermes_ctx* c) {
    if (!c) return "null context";
    return c->msg.c_str();
}

static int check_device_ptr(hermes_ctx* c, const void* p, const char* name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HERMES_ERR_ARG, "%s is not a valid pointer", name);
    }
    if (!(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) || a.device != c->device)
        return fail(c, HERMES_ERR_ARG, "%s is not device memory of device %d", name, c->device);
    return HERMES_OK;
}

int hermes_assign(hermes_ctx* c, const float* pos, const float* w, int64_t n, unsigned flags) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!pos) return fail(c, HERMES_ERR_ARG, "pos is NULL");
    if (n < 1) return fail(c, HERMES_ERR_ARG, "empty catalogue (n = %lld): the density contrast is undefined",
                           (long long)n);
    if (flags & ~(HERMES_DEVICE_PTR | HERMES_WRAP)) return fail(c, HERMES_ERR_ARG, "unknown flags 0x%x", flags);
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    c->have_field = false;
    cudaStream_t st = c->stream;
    const int N = c->N, p = c->p;
    const float* dpos = pos;
    const float* dw = w;
    if (flags & HERMES_DEVICE_PTR) {
        int r = check_device_ptr(c, pos, "pos");
        if (r) return r;
        if (w && (r = check_device_ptr(c, w, "w"))) return r;
    } else {
        if ((size_t)n > c->stage_cap) {
            dev_free(c->stage_pos);
            dev_free(c->stage_w);
            c->stage_pos = nullptr;
            c->stage_w = nullptr;
            c->stage_cap = 0;
            CK(dev_malloc((void**)&c->stage_pos, (size_t)n * 3 * sizeof(float)), "staging positions");
            CK(dev_malloc((void**)&c->stage_w, (size_t)n * sizeof(float)), "staging weights");
            c->stage_cap = (size_t)n;
        }
        CK(cudaMemcpyAsync(c->stage_pos, pos, (size_t)n * 3 * sizeof(float), cudaMemcpyDefault, st), "copy positions");
        if (w) CK(cudaMemcpyAsync(c->stage_w, w, (size_t)n * sizeof(float), cudaMemcpyDefault, st), "copy weights");
        dpos = c->stage_pos;
        dw = w ? c->stage_w : nullptr;
    }
    const size_t n3 = (size_t)N * N * N;
    const int p3 = p * p * p;
    const int nblk = 592;
    CK(grow_doubles(c->part, c->part_cap, (size_t)std::max(2, p3) * nblk), "partials");
    CK(grow_doubles(c->red, c->red_cap, 1024), "reduction buffer");
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    const float s = (float)((double)N / c->L);
    CK(scatter_tiled(c, dpos, dw, n, c->grid, s, (flags & HERMES_WRAP) ? 1 : 0, st), "scatter");
    CK(launch_weight_sums(dw, n, c->part, nblk, st, c->tracer), "weight sums");
    CK(launch_reduce_rows(c->part, 2, nblk, c->red, st, c->tracer), "reduce sums");
    CK(launch_selfpair(N, p, dpos, dw, n, s, c->part, nblk, st, c->tracer), "self-pair table");
    CK(launch_reduce_rows(c->part, p3, nblk, c->stab_d, st, c->tracer), "reduce self-pair");
    CK(launch_finish_field(c->red, c->stab_d, p3, c->stab_f, N, c->scal, st, c->tracer), "field scalars");
    CK(cudaMemcpyAsync(c->host_buf, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "read sums");
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "assign");
    if (herr) return fail(c, HERMES_ERR_RANGE, "a coordinate is outside [0, L] (u = x*N/L outside [0, N]) "
                                               "or a weight is not finite; use HERMES_WRAP to wrap");
    c->sum_w = c->host_buf[0];
    c->sum_w2 = c->host_buf[1];
    if (!(c->sum_w > 0.0) || !std::isfinite(c->sum_w))
        return fail(c, HERMES_ERR_RANGE, "sum of weights is %g; it must be positive", c->sum_w);
    if (c->have_randoms) {
        // Delta = (eps_D - alpha eps_R) / eps_bar_D, alpha = sum w_D / sum w_R; SN table S_D + alpha^2 S_R
        const double alpha = c->sum_w / c->sum_wr;
        const double inv_ebar = (double)n3 / c->sum_w;
        CK(launch_combine_randoms(c->grid, c->rgrid, n3, (float)alpha, (float)inv_ebar, c->stab_d, c->rstab_d,
                                  alpha * alpha, c->stab_f, p3, st, c->tracer),
           "difference field");
        CK(launch_delta_to_spec(N, c->grid, c->spec, c->scal, tables_of(c), st, c->tracer), "forward FFT");
    } else {
        CK(launch_forward(N, c->grid, c->spec, c->scal, tables_of(c), st, c->tracer), "forward FFT");
    }
    CK(cudaStreamSynchronize(st), "forward FFT");
    c->have_field = true;
    return HERMES_OK;
}

int64_t hermes_shell_table_len(int N) {
    if (!valid_N(N)) return -1;
    return table_len(N);
}

int hermes_shell_table_host(double L, int N, const double* r_edges, int n_edges, int l_max, double* out) {
    if (!valid_N(N) || !(L > 0) || !r_edges || !out || n_edges < 2 || l_max < 0 || l_max > 24) return HERMES_ERR_ARG;
    for (int e = 0; e < n_edges; ++e)
        if (!std::isfinite(r_edges[e]) || (e > 0 && !(r_edges[e] > r_edges[e - 1])) || r_edges[e] < 0)
            return HERMES_ERR_RANGE;
    build_shell_tables(L, table_len(N), r_edges, n_edges, l_max, out);
    return HERMES_OK;
}

namespace {
// Process-wide cache of built window tables in the device layout
// [(l*Q + q)*nbp + b], keyed by (L, N, edges); an entry built for a larger
// l_max serves a smaller one (the orders are the leading blocks).  Bounded in
// host memory, least recently used first out.
struct TableEntry {
    double L;
    int N;
    std::vector<double> edges;
    int l_max;
    std::shared_ptr<const std::vector<float>> data;
    uint64_t stamp;
};
std::mutex g_tab_mu;
std::vector<TableEntry> g_tabs;
uint64_t g_tab_clock = 0;
constexpr size_t kTableCacheBytes = (size_t)8 << 30;

std::shared_ptr<const std::vector<float>> table_lookup(double L, int N, const double* e, int ne, int l_max) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    TableEntry* best = nullptr;
    for (auto& t : g_tabs)
        if (t.L == L && t.N == N && t.l_max >= l_max && (int)t.edges.size() == ne &&
            std::equal(t.edges.begin(), t.edges.end(), e) && (!best || t.l_max < best->l_max))
            best = &t;
    if (!best) return nullptr;
    best->stamp = ++g_tab_clock;
    return best->data;
}

void table_insert(double L, int N, const double* e, int ne, int l_max, std::shared_ptr<const std::vector<float>> d) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    size_t total = d->size() * sizeof(float);
    for (auto& t : g_tabs) total += t.data->size() * sizeof(float);
    while (total > kTableCacheBytes && !g_tabs.empty()) {
        auto old = std::min_element(g_tabs.begin(), g_tabs.end(),
                                    [](const TableEntry& a, const TableEntry& b) { return a.stamp < b.stamp; });
        total -= old->data->size() * sizeof(float);
        g_tabs.erase(old);
    }
    if (d->size() * sizeof(float) <= kTableCacheBytes)
        g_tabs.push_back(TableEntry{L, N, std::vector<double>(e, e + ne), l_max, std::move(d), ++g_tab_clock});
}
}  // namespace

int hermes_window_shells(hermes_ctx* c, const double* r_edges, int n_edges, int l_max) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!r_edges) return fail(c, HERMES_ERR_ARG, "r_edges is NULL");
    if (n_edges < 2 || n_edges > 4097) return fail(c, HERMES_ERR_ARG, "n_edges = %d (need 2..4097)", n_edges);
    if (l_max < 0 || l_max > 24) return fail(c, HERMES_ERR_ARG, "l_max = %d (need 0..24)", l_max);
    for (int e = 0; e < n_edges; ++e) {
        if (!std::isfinite(r_edges[e]) || r_edges[e] < 0.0)
            return fail(c, HERMES_ERR_RANGE, "r_edges[%d] = %g is negative or not finite", e, r_edges[e]);
        if (e > 0 && !(r_edges[e] > r_edges[e - 1]))
            return fail(c, HERMES_ERR_RANGE, "r_edges must increase strictly (index %d)", e);
    }
    if (r_edges[n_edges - 1] > 0.5 * c->L)
        return fail(c, HERMES_ERR_RANGE, "largest edge %g exceeds L/2 = %g", r_edges[n_edges - 1], 0.5 * c->L);
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const int64_t Q = table_len(c->N);
    const int nb = n_edges - 1;
    const int nbp = (nb + 3) & ~3;
    const size_t count = (size_t)nb * (l_max + 1) * Q;
    const size_t count_dev = (size_t)nbp * (l_max + 1) * Q;
    std::shared_ptr<const std::vector<float>> tab = table_lookup(c->L, c->N, r_edges, n_edges, l_max);
    if (!tab) {
        std::shared_ptr<std::vector<float>> host32;
        std::vector<double> host;
        try {
            host.resize(count);
            host32 = std::make_shared<std::vector<float>>(count_dev, 0.0f);
        } catch (...) {
            return fail(c, HERMES_ERR_NOMEM, "host table of %zu entries", count);
        }
        build_shell_tables(c->L, Q, r_edges, n_edges, l_max, host.data());
        // device layout bin-fastest: [(l*Q + q)*nbp + b]
        for (int b = 0; b < nb; ++b)
            for (int l = 0; l <= l_max; ++l) {
                const double* src = host.data() + ((size_t)b * (l_max + 1) + l) * Q;
                float* dst = host32->data() + (size_t)l * Q * nbp + b;
                for (int64_t q = 0; q < Q; ++q) dst[(size_t)q * nbp] = (float)src[q];
            }
        tab = host32;
        table_insert(c->L, c->N, r_edges, n_edges, l_max, host32);
    }
    cudaStreamSynchronize(c->stream);
    dev_free(c->rad);
    c->rad = nullptr;
    c->n_bins = 0;
    CK(dev_malloc((void**)&c->rad, count_dev * sizeof(float)), "window tables");
    // the orders 0..l_max are the leading blocks of a cached table built for a larger l_max
    CK(upload(c->rad, tab->data(), count_dev * sizeof(float), c->stream), "upload window tables");
    c->edges.assign(r_edges, r_edges + n_edges);
    c->n_bins = nb;
    c->l_max = l_max;
    c->Q = Q;
    c->nbp = nbp;
    return HERMES_OK;
}

namespace {
// Radial-histogram terms of every window (entry a of idx, bin b) into
// out[a*nb + b] = c sum_q T_b(q) H_a(q) / N^6 (Eq. pair-counting-kspace):
//   self_only = 1: H is the self-pair histogram of the field whose float table is
//                  tb.stab (divide by eps_bar^2 for SN_b);
//   self_only = 0: H is the Parseval histogram (|delta^|^2 - S^/eps_bar^2), so out is xi.
// cyl = 0: idx are even orders l over the isotropic tables; cyl = 1: idx are
// line-of-sight bins j over the axisymmetric tables, or, with ring windows, the
// windows themselves (out[a] is then the single value of window idx[a]).  hist
// holds min(n, 8) * Q doubles.
cudaError_t enqueue_hist_terms(hermes_ctx* c, const Tables& tb, const double* scal, const int* idx, int n, int cyl,
                               int self_only, double* hist, double* out, cudaStream_t st, const Tracer& tr,
                               const float2* spec_override = nullptr) {
    const float* rad = cyl ? c->cyl_perp : c->rad;
    const int nbp = cyl ? c->cyl_nbp : c->nbp;
    const int64_t Q = cyl ? c->cyl_Q : c->Q;
    const int diag = cyl && c->cyl_ring;  // ring windows: one value per entry
    const int nb = diag ? 1 : (cyl ? c->cyl_nperp : c->n_bins);
    for (int a0 = 0; a0 < n; a0 += 8) {
        KsOrders ko;
        ko.n = std::min(8, n - a0);
        for (int k = 0; k < ko.n; ++k) ko.ell[k] = idx[a0 + k];
        ko.cyl = cyl;
        ko.par = c->cyl_par;
        ko.diag = diag;
        cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)ko.n * Q * sizeof(double), st);
        if (e != cudaSuccess) return e;
        const float2* spec = self_only ? nullptr : (spec_override ? spec_override : c->spec);
        if ((e = launch_kspace_hist(c->N, spec, tb, c->p, scal, ko, hist, Q, st, tr, self_only)) != cudaSuccess)
            return e;
        if ((e = launch_kspace_contract(rad, nbp, Q, ko, hist, c->N, out + (size_t)a0 * nb, nb, st, tr,
                                        self_only ? K_SN_CONTRACT : K_KSPACE_CONTRACT)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_selfpair_terms(hermes_ctx* c, const Tables& tb, const int* ells, int n_ells, double* hist,
                                   double* out, cudaStream_t st, const Tracer& tr) {
    return enqueue_hist_terms(c, tb, nullptr, ells, n_ells, 0, 1, hist, out, st, tr);
}

// RR of the random field for windows idx (isotropic orders or line-of-sight bins), by
// Parseval on its transform: out[a*nb + b] = c sum_q T_b(q) H_a(q) / N^6 with
// H the histogram of |eps^_R|^2 - S^_R (the randoms' self pairs removed); the caller
// scales by (N^3 / sum w_R)^2, which turns eps_R into alpha eps_R / eps_bar_D.
cudaError_t enqueue_rr_terms(hermes_ctx* c, const int* idx, int n, int cyl, double* hist, double* out,
                             cudaStream_t st, const Tracer& tr) {
    Tables tb = tables_of(c);
    tb.stab = c->rstab_f;
    return enqueue_hist_terms(c, tb, c->rscal, idx, n, cyl, 0, hist, out, st, tr, c->rspec);
}
}  // namespace

int hermes_xi_multipoles(hermes_ctx* c, const int* ells, int n_ells, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!ells || !out || n_ells < 1) return fail(c, HERMES_ERR_ARG, "ells/out NULL or n_ells < 1");
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->n_bins < 1) return fail(c, HERMES_ERR_STATE, "no bins: call hermes_window_shells first");
    for (int a = 0; a < n_ells; ++a) {
        if (ells[a] < 0 || ells[a] > c->l_max)
            return fail(c, HERMES_ERR_ARG, "l = %d outside 0..l_max = %d", ells[a], c->l_max);
        if (ells[a] & 1) return fail(c, HERMES_ERR_ARG, "odd l = %d vanishes for an auto-correlation", ells[a]);
    }
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, H = c->H, nb = c->n_bins;
    const int nwin = n_ells * nb;
    const size_t win_bytes = (size_t)N * N * H * sizeof(float2);
    const int S = (int)xi_window_S(N, nb);
    CK(grow(c->work, c->work_bytes, (size_t)S * win_bytes), "window work buffer");
    const int zb = inv_z_blocks(N);
    CK(grow_doubles(c->part, c->part_cap, std::max((size_t)S * zb, (size_t)std::min(n_ells, 8) * c->Q)), "partials");
    CK(grow_doubles(c->red, c->red_cap, (size_t)2 * nwin + nb), "reduction buffer");
    const Tables tb = tables_of(c);
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    // self-pair terms of all windows first (the histogram lives in the partials buffer)
    CK(enqueue_selfpair_terms(c, tb, ells, n_ells, c->part, c->red + nwin, st, c->tracer), "self-pair terms");
    // batches never cross an order: bins b0 .. b0+S-1 of one l (b0 a multiple of S)
    for (int a = 0; a < n_ells; ++a) {
        const int ell = ells[a];
        for (int b0 = 0; b0 < nb; b0 += S) {
            WinBatch wb;
            wb.S = std::min(S, nb - b0);
            wb.tab = c->rad + (size_t)ell * c->Q * c->nbp + b0;
            wb.nbp = c->nbp;
            wb.ell = ell;
            wb.scale = (float)((2 * ell + 1) * (((ell / 2) & 1) ? -1 : 1));  // (2l+1) i^l, l even
            const int w0 = a * nb + b0;
            double* dd_part = c->part;
            CK(launch_inverse_xi(N, c->spec, c->work, c->grid, wb, tb, dd_part, c->err, st, c->tracer),
               "inverse passes");
            CK(launch_reduce_rows(dd_part, wb.S, zb, c->red + w0, st, c->tracer), "reduce contractions");
        }
    }
    const int nrr = c->have_randoms ? nb : 0;  // RR of the l = 0 window of every bin
    if (nrr) {
        const int zero = 0;
        CK(enqueue_rr_terms(c, &zero, 1, 0, c->part, c->red + 2 * nwin, st, c->tracer), "random pairs");
    }
    CK(ensure_host(c, (size_t)2 * nwin + nrr + 1) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation,
       "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(2 * nwin + nrr) * sizeof(double), cudaMemcpyDeviceToHost, st),
       "read xi");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + (size_t)2 * nwin + nrr);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "xi");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
    const double n3 = (double)N * N * N;
    const double n6 = n3 * n3;
    const double eps_bar = c->sum_w / n3;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int widx = 0; widx < nwin; ++widx) {
        const double dd = c->host_buf[widx] / n6;
        const double sn = c->host_buf[nwin + widx] / (eps_bar * eps_bar);  // already / N^6
        // Eq. xi-deltaDD-over-RR: RR = 1 for analytic uniform randoms; xi_l divides by RR_0
        const double rr = nrr ? c->host_buf[2 * nwin + widx % nb] * rr_scale : 1.0;
        out[widx] = (dd - sn) / rr;
    }
    return HERMES_OK;
}

int hermes_xi_multipoles_kspace(hermes_ctx* c, const int* ells, int n_ells, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!ells || !out || n_ells < 1 || n_ells > 8) return fail(c, HERMES_ERR_ARG, "ells/out NULL or n_ells not in 1..8");
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->n_bins < 1) return fail(c, HERMES_ERR_STATE, "no bins: call hermes_window_shells first");
    KsOrders ko;
    ko.n = n_ells;
    for (int a = 0; a < n_ells; ++a) {
        if (ells[a] < 0 || ells[a] > c->l_max)
            return fail(c, HERMES_ERR_ARG, "l = %d outside 0..l_max = %d", ells[a], c->l_max);
        if (ells[a] & 1) return fail(c, HERMES_ERR_ARG, "odd l = %d vanishes for an auto-correlation", ells[a]);
        ko.ell[a] = ells[a];
    }
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int nb = c->n_bins;
    const size_t nh = (size_t)n_ells * c->Q;
    CK(grow_doubles(c->part, c->part_cap, nh), "histogram");
    CK(grow_doubles(c->red, c->red_cap, (size_t)n_ells * nb + nb), "reduction buffer");  // + RR per bin
    CK(cudaMemsetAsync(c->part, 0, nh * sizeof(double), st), "clear histogram");
    CK(launch_kspace_hist(c->N, c->spec, tables_of(c), c->p, c->scal, ko, c->part, c->Q, st, c->tracer),
       "k-space histogram");
    CK(launch_kspace_contract(c->rad, c->nbp, c->Q, ko, c->part, c->N, c->red, nb, st, c->tracer), "k-space sums");
    const int nrr = c->have_randoms ? nb : 0;
    if (nrr) {
        const int zero = 0;
        CK(enqueue_rr_terms(c, &zero, 1, 0, c->part, c->red + (size_t)n_ells * nb, st, c->tracer), "random pairs");
    }
    CK(ensure_host(c, (size_t)n_ells * nb + nrr) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation,
       "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(n_ells * nb + nrr) * sizeof(double), cudaMemcpyDeviceToHost,
                       st),
       "read xi");
    CK(cudaStreamSynchronize(st), "xi (k-space)");
    const double n3 = (double)c->N * c->N * c->N;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int i = 0; i < n_ells * nb; ++i)
        out[i] = c->host_buf[i] / (nrr ? c->host_buf[n_ells * nb + i % nb] * rr_scale : 1.0);
    return HERMES_OK;
}

int hermes_xi(hermes_ctx* c, double* out) {
    const int zero = 0;
    return hermes_xi_multipoles(c, &zero, 1, out);
}

namespace {
// Centred cardinal B-spline M_p(x) (unit integral, support |x| < p/2) by the recursion of the
// uniform B-spline, M_1 = the box [-1/2, 1/2) and
// M_p(x) = ((x + p/2) M_{p-1}(x + 1/2) + (p/2 - x) M_{p-1}(x - 1/2)) / (p - 1).
double bspline_host(int p, double x) {
    if (p == 1) return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    if (std::fabs(x) >= 0.5 * p) return 0.0;
    return ((x + 0.5 * p) * bspline_host(p - 1, x + 0.5) + (0.5 * p - x) * bspline_host(p - 1, x - 0.5)) / (p - 1);
}

// n-point Gauss-Legendre nodes and weights on [0, 1]: the roots of P_n by Newton's method
// from the estimates cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the three-term recurrence,
// weights 2 / ((1 - z^2) P_n'(z)^2), mapped from [-1, 1].
void gauss_legendre01(int n, double* t, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            dp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-15) break;
        }
        t[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}
}  // namespace

// Warps per block of the monopole Gram for 9 to 16 bins: 2 (each a diagonal tile and half of
// the off-diagonal one) unless HERMES_DDD_WARPS=3 (one tile per warp; kept for comparison).
static int ddd_gram_warps() {
    const char* e = getenv("HERMES_DDD_WARPS");
    return (e && e[0] == '3') ? 3 : 2;
}

int hermes_ddd_monopole(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!out) return fail(c, HERMES_ERR_ARG, "out is NULL");
    if (c->p > 4)
        return fail(c, HERMES_ERR_ARG, "the monopole's sample kernels are built for orders p <= 4 (context p = %d)",
                    c->p);
    if (c->have_randoms)
        return fail(c, HERMES_ERR_STATE, "the monopole uses analytic uniform randoms: call hermes_clear_randoms and "
                                         "hermes_assign first");
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->n_bins < 1) return fail(c, HERMES_ERR_STATE, "no bins: call hermes_window_shells first");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, H = c->H, nb = c->n_bins, p = c->p, nf = nb + 1;
    const size_t n3 = (size_t)N * N * N;
    // The Gram runs over field-slot sets of delta and up to 16 bins: all bins at once up to 16
    // bins (one warp up to 8 bins; above, two warps, each a diagonal 8 x 8 tile and half of the
    // off-diagonal one, or three with one tile each); beyond, one run per pair of 8-bin blocks
    // I <= J (one warp: the upper triangle of block I, or the block (I, J)).
    struct Run {
        int nw, I, J, tile0;
    };
    std::vector<Run> runs;
    if (nb <= 16) {
        runs.push_back({nb <= 8 ? 1 : ddd_gram_warps(), 0, 1, 0});
    } else {
        const int B = (nb + 7) / 8;
        for (int I = 0; I < B; ++I)
            for (int J = I; J < B; ++J) runs.push_back({1, I, J, I == J ? 0 : 1});
    }
    std::vector<size_t> part_off(runs.size() + 1, 0);
    for (size_t r = 0; r < runs.size(); ++r)
        part_off[r + 1] = part_off[r] + (size_t)ddd_gram_blocks(N, runs[r].nw) * 3 * 64;
    const size_t npart = part_off.back();
    // work: up to 16 half spectra; F = [delta, f_0 .. f_{nb-1}] and its filtered copy Y, N^3 floats each
    const int wmax = std::min(nb, 16);
    CK(grow(c->work, c->work_bytes, (size_t)wmax * N * N * H * sizeof(float2)), "window work buffer");
    CK(grow(c->zfields, c->zfields_bytes, (size_t)2 * nf * n3 * sizeof(float)), "monopole fields");
    float* F = reinterpret_cast<float*>(c->zfields);
    float* Y = F + (size_t)nf * n3;
    CK(grow_doubles(c->part, c->part_cap, npart), "partials");
    const Tables tb = tables_of(c);
    CK(cudaMemcpyAsync(F, c->grid, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy delta");
    // f_b = iFT[delta^ <j_0>_b Phi^] / N^3: the l = 0 shell windows of the xi tables, 16 bins a batch
    for (int b0 = 0; b0 < nb; b0 += 16) {
        WinBatch wb;
        wb.S = std::min(16, nb - b0);
        wb.tab = c->rad + b0;
        wb.nbp = c->nbp;
        wb.ell = 0;
        wb.scale = 1.0f;
        CK(launch_filtered_fields(N, c->spec, c->work, F + (size_t)(1 + b0) * n3, wb, tb, st, c->tracer),
           "shell fields");
    }
    // knot cells [c + o, c + o + 1) (o = 0 for even p, -1/2 for odd p); a spline field at
    // u = c + o + t reads the coefficients c + j0 + j, j < p, with weights M_p(t + o - j0 - j)
    const int ng = ddd_samples(p);
    double t[DDD_MAX_SAMPLES], w[DDD_MAX_SAMPLES], B[DDD_MAX_SAMPLES][8] = {};
    gauss_legendre01(ng, t, w);
    const double o = (p & 1) ? -0.5 : 0.0;
    const int j0 = (p & 1) ? -(p - 1) / 2 : 1 - p / 2;
    std::vector<DddTaps> tx(runs.size());
    for (size_t r = 0; r < runs.size(); ++r) {
        DddTaps& d = tx[r];
        d = DddTaps{};
        for (int a = 0; a < ng; ++a) {
            for (int j = 0; j < p; ++j) {
                B[a][j] = bspline_host(p, t[a] + o - j0 - j);
                d.bx[a][j] = (float)B[a][j];
            }
            d.wx[a] = (float)w[a];
        }
        d.j0 = j0;
        d.tile0 = runs[r].tile0;
        d.fld[0] = 0;
        for (int k = 0; k < 8; ++k) {
            const int br = 8 * runs[r].I + k, bc = 8 * runs[r].J + k;
            d.fld[1 + k] = br < nb ? 1 + br : -1;
            d.fld[9 + k] = (bc < nb && (runs[r].nw > 1 || runs[r].tile0 == 1)) ? 1 + bc : -1;
        }
    }
    CK(cudaMemsetAsync(c->part, 0, npart * sizeof(double), st), "clear partials");
    for (int gz = 0; gz < ng; ++gz) {
        for (int gy = 0; gy < ng; ++gy) {
            DddYZ yz{};
            for (int j = 0; j < p; ++j) {
                yz.by[j] = (float)B[gy][j];
                yz.bz[j] = (float)B[gz][j];
            }
            yz.j0 = j0;
            CK(launch_ddd_filter_yz(N, p, F, Y, nf, yz, st, c->tracer), "sample filters");
            for (size_t r = 0; r < runs.size(); ++r) {
                tx[r].wyz = w[gy] * w[gz];
                CK(launch_ddd_gram(N, p, Y, runs[r].nw, tx[r], c->part + part_off[r], st, c->tracer),
                   "monopole Gram");
            }
        }
    }
    CK(ensure_host(c, npart) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->part, npart * sizeof(double), cudaMemcpyDeviceToHost, st), "read Gram");
    CK(cudaStreamSynchronize(st), "monopole");
    for (int i = 0; i < nb * nb; ++i) out[i] = 0.0;
    for (size_t r = 0; r < runs.size(); ++r) {
        const int gb = ddd_gram_blocks(N, runs[r].nw);
        const bool all3 = runs[r].nw > 1;  // tiles 0, 1, 2 in slots 0, 1, 2
        const int ntile = all3 ? 3 : 1;
        for (int ts = 0; ts < ntile; ++ts) {
            // tile (row block, column block) of entries 8 a + b
            const int tile = all3 ? ts : runs[r].tile0;
            const int rb = all3 ? (tile == 2 ? 1 : 0) : runs[r].I;
            const int cbk = all3 ? (tile == 0 ? 0 : 1) : (tile == 0 ? runs[r].I : runs[r].J);
            const bool diag = tile != 1;
            for (int k = 0; k < 64; ++k) {
                const int b1 = 8 * rb + k / 8, b2 = 8 * cbk + k % 8;
                if (b1 >= nb || b2 >= nb || (diag && k % 8 < k / 8)) continue;
                double sum = 0.0;
                for (int blk = 0; blk < gb; ++blk) sum += c->host_buf[part_off[r] + ((size_t)blk * 3 + ts) * 64 + k];
                out[b1 * nb + b2] = out[b2 * nb + b1] = sum / (double)n3;
            }
        }
    }
    return HERMES_OK;
}

int hermes_zeta_multipoles(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!out) return fail(c, HERMES_ERR_ARG, "out is NULL");
    if (c->have_randoms)
        return fail(c, HERMES_ERR_STATE, "zeta_l uses analytic uniform randoms: call hermes_clear_randoms and "
                                         "hermes_assign first");
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->n_bins < 1) return fail(c, HERMES_ERR_STATE, "no bins: call hermes_window_shells first");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, nb = c->n_bins, LM = c->l_max + 1;
    const size_t n3 = (size_t)N * N * N;
    // Up to 16 bins go through the passes together.  More bins are taken in blocks of 8:
    // every pair of blocks (I <= J) runs as one batch of at most 16 bins, and each Gram
    // entry is kept from the run of its two bins' blocks.
    struct Run {
        int I, J, S;  // J = -1: block I alone (or all bins when nb <= 16)
    };
    std::vector<Run> runs;
    const int nblk = (nb + 7) / 8;
    auto bsize = [&](int I) { return std::min(8, nb - 8 * I); };
    if (nb <= 16) {
        runs.push_back({0, -1, nb});
    } else {
        for (int I = 0; I < nblk; ++I)
            for (int J = I; J < nblk; ++J) runs.push_back({I, J == I ? -1 : J, bsize(I) + (J == I ? 0 : bsize(J))});
    }
    const int nruns = (int)runs.size();
    const int smax = std::min(nb, 16);
    CK(grow(c->zfields, c->zfields_bytes, (size_t)smax * n3 * sizeof(float2)), "harmonic fields");
    const int zb = zeta_z_blocks(N);
    CK(grow_doubles(c->part, c->part_cap, (size_t)256 * zb), "partials");
    const int nlm = LM * (LM + 1) / 2;
    CK(grow_doubles(c->red, c->red_cap, (size_t)256 * nlm * nruns), "reduction buffer");
    const Tables tb = tables_of(c);
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    int lm = 0;
    for (int ell = 0; ell < LM; ++ell) {
        for (int m = 0; m <= ell; ++m, ++lm) {
            double norm = std::sqrt((2.0 * ell + 1.0) / (4.0 * M_PI) * std::tgamma(ell - m + 1.0) /
                                    std::tgamma(ell + m + 1.0));
            norm *= ((m & 1) ? -1.0 : 1.0) * dfact2(2 * m - 1);
            const float* tab_l = c->rad + (size_t)ell * c->Q * c->nbp;
            for (int r = 0; r < nruns; ++r) {
                HarmBatch hb;
                hb.S = runs[r].S;
                hb.ell = ell;
                hb.m = m;
                hb.ylm_norm = (float)(4.0 * M_PI * norm);
                hb.tab = tab_l + 8 * runs[r].I;
                hb.tab2 = runs[r].J >= 0 ? tab_l + 8 * runs[r].J : nullptr;
                hb.nbp = c->nbp;
                CK(launch_zeta_lm(N, c->spec, c->zfields, c->grid, hb, tb, c->part, c->err, st, c->tracer),
                   "harmonic fields");
                CK(launch_reduce_rows(c->part, 256, zb, c->red + (size_t)256 * ((size_t)lm * nruns + r), st,
                                      c->tracer),
                   "reduce Gram");
            }
        }
    }
    const size_t nred = (size_t)256 * nlm * nruns;
    CK(ensure_host(c, nred + 1) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, nred * sizeof(double), cudaMemcpyDeviceToHost, st), "read Gram");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + nred);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "zeta");
    if (*hflag & 2u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on the tensor-core pipeline gave up");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
    const double nn = (double)N;
    const double scale = 1.0 / (4.0 * M_PI * std::pow(nn, 9));
    for (size_t e = 0; e < (size_t)LM * nb * nb; ++e) out[e] = 0.0;
    lm = 0;
    for (int ell = 0; ell < LM; ++ell) {
        double* o = out + (size_t)ell * nb * nb;
        for (int m = 0; m <= ell; ++m, ++lm) {
            const double wm = (m == 0) ? 1.0 : 2.0;
            for (int r = 0; r < nruns; ++r) {
                const double* G = c->host_buf + (size_t)256 * ((size_t)lm * nruns + r);
                const Run& ru = runs[r];
                auto glob = [&](int i) { return (ru.J >= 0 && i >= 8) ? 8 * ru.J + (i - 8) : 8 * ru.I + i; };
                for (int i1 = 0; i1 < ru.S; ++i1)
                    for (int i2 = i1; i2 < ru.S; ++i2) {
                        // a pair run keeps only its cross entries (block I x block J)
                        if (ru.J >= 0 && !(i1 < 8 && i2 >= 8)) continue;
                        const int b1 = glob(i1), b2 = glob(i2);
                        const double v = wm * G[i1 * 16 + i2] * scale;  // upper triangle, exact symmetry
                        o[(size_t)b1 * nb + b2] += v;
                        if (b1 != b2) o[(size_t)b2 * nb + b1] += v;
                    }
            }
        }
    }
    return HERMES_OK;
}

int hermes_debug_get_delta(hermes_ctx* c, float* host_out) {
    if (check_ctx(c) || !host_out) return HERMES_ERR_ARG;
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const size_t n3 = (size_t)c->N * c->N * c->N;
    CK(cudaMemcpyAsync(host_out, c->grid, n3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "read delta");
    CK(cudaStreamSynchronize(c->stream), "read delta");
    return HERMES_OK;
}

int hermes_debug_get_spectrum(hermes_ctx* c, float* host_out) {
    if (check_ctx(c) || !host_out) return HERMES_ERR_ARG;
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const size_t cnt = (size_t)c->N * c->N * c->H;
    CK(cudaMemcpyAsync(host_out, c->spec, cnt * sizeof(float2), cudaMemcpyDeviceToHost, c->stream), "read spectrum");
    CK(cudaStreamSynchronize(c->stream), "read spectrum");
    return HERMES_OK;
}

int hermes_debug_set_delta(hermes_ctx* c, const float* host_delta) {
    if (check_ctx(c) || !host_delta) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const size_t n3 = (size_t)c->N * c->N * c->N;
    c->have_field = false;
    CK(cudaMemcpyAsync(c->grid, host_delta, n3 * sizeof(float), cudaMemcpyDefault, c->stream), "write delta");
    CK(cudaMemsetAsync(c->stab_f, 0, 512 * sizeof(float), c->stream), "clear self-pair");
    CK(cudaMemsetAsync(c->stab_d, 0, 512 * sizeof(double), c->stream), "clear self-pair");
    const double scal_host[3] = {(double)n3, 0.0, 1.0};  // sum w = N^3, eps_bar = 1
    CK(cudaMemcpyAsync(c->scal, scal_host, sizeof(scal_host), cudaMemcpyHostToDevice, c->stream), "field scalars");
    CK(launch_delta_to_spec(c->N, c->grid, c->spec, c->scal, tables_of(c), c->stream, c->tracer), "forward FFT");
    CK(cudaStreamSynchronize(c->stream), "set delta");
    c->sum_w = (double)n3;  // eps_bar = 1
    c->sum_w2 = 0.0;
    c->have_field = true;
    return HERMES_OK;
}

int hermes_debug_nodes(hermes_ctx* c, const float* host_pos, int64_t n, unsigned flags, int* host_first,
                       float* host_wts) {
    if (check_ctx(c) || !host_pos || !host_first || !host_wts || n < 1) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int p = c->p;
    float* dpos = nullptr;
    int* dfirst = nullptr;
    float* dw = nullptr;
    int rc = HERMES_OK;
    unsigned herr = 0;
    cudaError_t e = dev_malloc((void**)&dpos, (size_t)n * 3 * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc((void**)&dfirst, (size_t)n * 3 * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc((void**)&dw, (size_t)n * 3 * p * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpos, host_pos, (size_t)n * 3 * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = launch_nodes(c->N, p, dpos, n, (float)((double)c->N / c->L), (flags & HERMES_WRAP) ? 1 : 0, dfirst, dw,
                         c->err, st, c->tracer);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_first, dfirst, (size_t)n * 3 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_wts, dw, (size_t)n * 3 * p * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "node rule");
    else if (herr) rc = fail(c, HERMES_ERR_RANGE, "a coordinate is outside the accepted range");
    dev_free(dpos);
    dev_free(dfirst);
    dev_free(dw);
    return rc;
}

static const char* const kKernelNames[K_COUNT] = {
    "scatter", "weight_sums", "selfpair", "reduce", "finish_field", "fwd_z_r2c", "fwd_y", "fwd_x",
    "inv_x_window", "inv_y", "inv_z_c2r_contract", "zeta_x", "zeta_y", "zeta_z_gram", "nodes",
    "inv_yz_contract", "zeta_z_gram_tc", "kspace_hist", "kspace_contract", "batch_graph", "selfpair_hist", "selfpair_contract", "combine_randoms", "inv_z_store", "gather_marks", "wait_check",
    "ddd_filter", "ddd_gram"};

int hermes_trace_enable(hermes_ctx* c, int on) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    trace_collect(c);
    for (int i = 0; i < K_COUNT; ++i) {
        c->trace_ms[i] = 0.0;
        c->trace_n[i] = 0;
    }
    c->trace_on = on != 0;
    return HERMES_OK;
}

int hermes_trace_read(hermes_ctx* c, double* ms, int64_t* launches, int n) {
    if (check_ctx(c) || n < 0) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    trace_collect(c);
    for (int i = 0; i < n && i < K_COUNT; ++i) {
        if (ms) ms[i] = c->trace_ms[i];
        if (launches) launches[i] = c->trace_n[i];
    }
    for (int i = 0; i < K_COUNT; ++i) {
        c->trace_ms[i] = 0.0;
        c->trace_n[i] = 0;
    }
    return K_COUNT;
}

const char* hermes_kernel_name(int id) {
    if (id < 0 || id >= K_COUNT) return "";
    return kKernelNames[id];
}

int64_t hermes_launch_count(const hermes_ctx* c) { return c ? c->launches : -1; }

int hermes_debug_bounded_wait(hermes_ctx* c) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    CK(launch_wait_unarrived(c->err, st, c->tracer), "bounded wait");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "bounded wait");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on an mbarrier gave up");
    return HERMES_OK;
}

int hermes_debug_fail_allocs(int count) { return g_fail_allocs.exchange(count < 0 ? 0 : count); }

int hermes_debug_get_sums(hermes_ctx* c, double* sums2, double* selfpair) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    if (sums2) {
        sums2[0] = c->sum_w;
        sums2[1] = c->sum_w2;
    }
    if (selfpair) {
        const int p3 = c->p * c->p * c->p;
        CK(cudaMemcpyAsync(selfpair, c->stab_d, p3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read table");
        CK(cudaStreamSynchronize(c->stream), "read table");
    }
    return HERMES_OK;
}

}  // extern "C"

// ===========================================================================
// hermes_assign_noalloc: hermes_assign for callers that must not allocate.
//
// The per-block partial sums of the weight and self-pair reductions live in
// this file-scope device array instead of context buffers that grow on demand.
// In host code the name g_assign_scratch is only a host-side stand-in: its
// device address is looked up once per device with cudaGetSymbolAddress and
// passed to the kernels.  Every context and every call on a device shares the
// array, so calls whose work overlaps on the GPU race on it.
namespace {
constexpr int kNoallocBlocks = 148;
constexpr size_t kNoallocDoubles = 32768;  // 256 KiB
static __device__ __align__(256) double g_assign_scratch[kNoallocDoubles];
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

int noalloc_scratch(hermes_ctx* c, double** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (c->device < 0 || c->device >= 256) return fail(c, HERMES_ERR_ARG, "device ordinal %d out of range", c->device);
    if (!g_noalloc_ptr[c->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_assign_scratch);  // the calling device is current
        if (e != cudaSuccess) return cuda_fail(c, e, "address of the static scratch array");
        g_noalloc_ptr[c->device] = (double*)p;
    }
    *out = g_noalloc_ptr[c->device];
    return HERMES_OK;
}

void count_only_mark(void* vc, int, int phase, cudaStream_t) {
    if (phase == 0) ++((hermes_ctx*)vc)->launches;
}
}  // namespace

extern "C" int hermes_assign_noalloc(hermes_ctx* c, const float* pos, const float* w, int64_t n, unsigned flags) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!pos) return fail(c, HERMES_ERR_ARG, "pos is NULL");
    if (n < 1) return fail(c, HERMES_ERR_ARG, "empty catalogue (n = %lld): the density contrast is undefined",
                           (long long)n);
    if (flags & ~(HERMES_DEVICE_PTR | HERMES_WRAP)) return fail(c, HERMES_ERR_ARG, "unknown flags 0x%x", flags);
    if (c->have_randoms)
        return fail(c, HERMES_ERR_STATE, "hermes_assign_noalloc builds analytic-random fields only; "
                                         "use hermes_assign with explicit randoms");
    const int N = c->N, p = c->p;
    const int p3 = p * p * p;
    const size_t need = 2 + (size_t)std::max(2, p3) * kNoallocBlocks;
    if (need > kNoallocDoubles)
        return fail(c, HERMES_ERR_ARG,
                    "hermes_assign_noalloc: its fixed scratch holds %zu doubles, order p = %d needs %zu "
                    "(p <= 6 fits); use hermes_assign", kNoallocDoubles, p, need);
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    int r = check_device_ptr(c, pos, "pos");
    if (r) return r;
    if (w && (r = check_device_ptr(c, w, "w"))) return r;
    double* scratch = nullptr;
    if ((r = noalloc_scratch(c, &scratch))) return r;
    double* sums = scratch;      // [2] reduced sum w, sum w^2
    double* part = scratch + 2;  // [max(2,p^3)][kNoallocBlocks] partials, fully overwritten
    c->have_field = false;
    cudaStream_t st = c->stream;
    const Tracer tr{c, count_only_mark};
    const size_t n3 = (size_t)N * N * N;
    CK(cudaMemsetAsync(c->grid, 0, n3 * sizeof(float), st), "clear grid");
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    const float s = (float)((double)N / c->L);
    CK(launch_scatter(N, p, pos, w, n, c->grid, s, (flags & HERMES_WRAP) ? 1 : 0, c->err, st, tr), "scatter");
    CK(launch_weight_sums(w, n, part, kNoallocBlocks, st, tr), "weight sums");
    CK(launch_reduce_rows(part, 2, kNoallocBlocks, sums, st, tr), "reduce sums");
    CK(launch_selfpair(N, p, pos, w, n, s, part, kNoallocBlocks, st, tr), "self-pair table");
    CK(launch_reduce_rows(part, p3, kNoallocBlocks, c->stab_d, st, tr), "reduce self-pair");
    CK(launch_finish_field(sums, c->stab_d, p3, c->stab_f, N, c->scal, st, tr), "field scalars");
    // both read-backs land in the pinned buffer allocated when the context was created
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + 2);
    CK(cudaMemcpyAsync(c->host_buf, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "read sums");
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "assign");
    if (*hflag) return fail(c, HERMES_ERR_RANGE, "a coordinate is outside [0, L] (u = x*N/L outside [0, N]) "
                                               "or a weight is not finite; use HERMES_WRAP to wrap");
    c->sum_w = c->host_buf[0];
    c->sum_w2 = c->host_buf[1];
    if (!(c->sum_w > 0.0) || !std::isfinite(c->sum_w))
        return fail(c, HERMES_ERR_RANGE, "sum of weights is %g; it must be positive", c->sum_w);
    CK(launch_forward(N, c->grid, c->spec, c->scal, tables_of(c), st, tr), "forward FFT");
    CK(cudaStreamSynchronize(st), "forward FFT");
    c->have_field = true;
    return HERMES_OK;
}

// ---------------------------------------------------------------------------
// Batched measurements: many catalogues on the same grid and windows.
//
// Every pass is one launch over all catalogues of a chunk (the catalogue is a
// grid dimension of each kernel); the whole measurement (scatter .. final xi)
// is captured once into a CUDA graph per shape and replayed on later calls.
// Windows per launch (S) and catalogues per launch (C) are chosen by timing the
// inverse passes on the live spectra the first time a shape is seen; the
// choice is cached for the process.

struct BatchPlan {
    int S = 0, C = 0;
};

struct BatchState {
    float* pos = nullptr;
    float* w = nullptr;
    size_t pts_cap = 0;                // points
    int64_t* offs = nullptr;           // [MAX_CATALOGUES + 1]
    float* grid = nullptr;             // [cat][N^3]
    float2* spec = nullptr;            // [cat][N*N*H]
    int cat_cap = 0;
    double* scal = nullptr;            // [cat][SCAL_STRIDE]
    float* stab_f = nullptr;           // [cat][STAB_STRIDE]
    double* sums = nullptr;            // [cat][2]
    double* sp = nullptr;              // [cat][512]
    double* part = nullptr;
    size_t part_cap = 0;               // doubles
    double* res = nullptr;             // dd, sn, xi: [3][cat][nwin]
    size_t res_cap = 0;                // doubles
    float2* work = nullptr;
    size_t work_bytes = 0;
    BatchPlan forced, last;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> key;
    int64_t graph_kernels = 0;
    int64_t graph_launches = 0;        // replays of the cached graph (for tests)
    std::vector<double> tune_ms;       // [candidate] = {S, C, ms per catalogue-window}
};

void batch_free(BatchState* b) {
    if (!b) return;
    dev_free(b->pos);
    dev_free(b->w);
    dev_free(b->offs);
    dev_free(b->grid);
    dev_free(b->spec);
    dev_free(b->scal);
    dev_free(b->stab_f);
    dev_free(b->sums);
    dev_free(b->sp);
    dev_free(b->part);
    dev_free(b->res);
    dev_free(b->work);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaGetLastError();
    delete b;
}

namespace {

std::mutex g_plan_mu;
std::map<std::vector<int64_t>, BatchPlan> g_plans;  // (device, N, p, ncat, nb, n_ells) -> plan

struct BatchJob {
    int ncat;
    int64_t n_total;
    bool has_w, wrap;
    std::vector<int> ells;
    BatchPlan plan;
};

int batch_nblk(int ncat) { return std::max(8, std::min(592, 2048 / ncat)); }

size_t batch_work_limit(const hermes_ctx* c) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return (size_t)8 << 30;
    }
    size_t have = free_b + c->batch->work_bytes;
    return std::min<size_t>((size_t)32 << 30, have / 3);
}

// Partials of the inverse passes for C catalogues x S windows.
size_t batch_part_need(int N, int S, int C) {
    return (size_t)C * S * (size_t)std::max(inv_z_blocks(N), inv_z_blocks_plain(N));
}

cudaError_t batch_grow(hermes_ctx* c, const BatchJob& j, int S_max, int C_max) {
    BatchState* b = c->batch;
    const int N = c->N;
    const size_t n3 = (size_t)N * N * N;
    cudaError_t e;
    if ((size_t)j.n_total > b->pts_cap) {
        dev_free(b->pos);
        dev_free(b->w);
        b->pos = nullptr;
        b->w = nullptr;
        b->pts_cap = 0;
        if ((e = dev_malloc((void**)&b->pos, (size_t)j.n_total * 3 * sizeof(float))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->w, (size_t)j.n_total * sizeof(float))) != cudaSuccess) return e;
        b->pts_cap = (size_t)j.n_total;
    }
    if (!b->offs && (e = dev_malloc((void**)&b->offs, (MAX_CATALOGUES + 1) * sizeof(int64_t))) != cudaSuccess) return e;
    if (j.ncat > b->cat_cap) {
        dev_free(b->grid);
        dev_free(b->spec);
        dev_free(b->scal);
        dev_free(b->stab_f);
        dev_free(b->sums);
        dev_free(b->sp);
        b->grid = nullptr;
        b->spec = nullptr;
        b->scal = nullptr;
        b->stab_f = nullptr;
        b->sums = nullptr;
        b->sp = nullptr;
        b->cat_cap = 0;
        const size_t k = (size_t)j.ncat;
        if ((e = dev_malloc((void**)&b->grid, k * n3 * sizeof(float))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->spec, k * (size_t)N * N * (N / 2) * sizeof(float2))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->scal, k * SCAL_STRIDE * sizeof(double))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->stab_f, k * STAB_STRIDE * sizeof(float))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->sums, k * 2 * sizeof(double))) != cudaSuccess) return e;
        if ((e = dev_malloc((void**)&b->sp, k * 512 * sizeof(double))) != cudaSuccess) return e;
        b->cat_cap = j.ncat;
    }
    const int p3 = c->p * c->p * c->p;
    const size_t nblk = (size_t)batch_nblk(j.ncat);
    size_t part_need = std::max<size_t>((size_t)j.ncat * std::max(2, p3) * nblk, batch_part_need(N, S_max, C_max));
    part_need = std::max(part_need, (size_t)std::min<size_t>(j.ells.size(), 8) * c->Q);  // self-pair histogram
    if ((e = grow_doubles(b->part, b->part_cap, part_need)) != cudaSuccess) return e;
    const size_t nwin = j.ells.size() * (size_t)c->n_bins;
    if ((e = grow_doubles(b->res, b->res_cap, 3 * (size_t)j.ncat * nwin)) != cudaSuccess) return e;
    const size_t win_bytes = (size_t)N * N * (N / 2) * sizeof(float2);
    return grow(b->work, b->work_bytes, (size_t)S_max * C_max * win_bytes);
}

// Scatter, sums, self-pair tables and forward transforms of every catalogue.
cudaError_t batch_enqueue_assign(hermes_ctx* c, const BatchJob& j, cudaStream_t st, const Tracer& tr) {
    BatchState* b = c->batch;
    const int N = c->N, p = c->p, p3 = p * p * p;
    const size_t n3 = (size_t)N * N * N;
    const int nblk = batch_nblk(j.ncat);
    const float s = (float)((double)N / c->L);
    const float* w = j.has_w ? b->w : nullptr;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->err, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    // groups of catalogues whose grids share about half of L2: each group's
    // clear and scatter atomics then stay on chip
    const size_t grid_bytes = n3 * sizeof(float);
    const int group = (int)std::max<size_t>(1, ((size_t)48 << 20) / grid_bytes);
    for (int c0 = 0; c0 < j.ncat; c0 += group) {
        const int c1 = std::min(j.ncat, c0 + group);
        if ((e = cudaMemsetAsync(b->grid + (size_t)c0 * n3, 0, (size_t)(c1 - c0) * grid_bytes, st)) != cudaSuccess)
            return e;
        if ((e = launch_scatter_batch(N, p, b->pos, w, b->offs, c0, c1, j.n_total, b->grid, s, j.wrap ? 1 : 0, c->err,
                                      st, tr)) != cudaSuccess)
            return e;
    }
    if ((e = launch_weight_sums(w, j.n_total, b->part, nblk, st, tr, b->offs, j.ncat)) != cudaSuccess) return e;
    if ((e = launch_reduce_rows(b->part, j.ncat * 2, nblk, b->sums, st, tr)) != cudaSuccess) return e;
    if ((e = launch_selfpair(N, p, b->pos, w, j.n_total, s, b->part, nblk, st, tr, b->offs, j.ncat)) != cudaSuccess)
        return e;
    if ((e = launch_reduce_rows(b->part, j.ncat * p3, nblk, b->sp, st, tr)) != cudaSuccess) return e;
    if ((e = launch_finish_batch(b->sums, b->sp, p3, b->stab_f, N, b->scal, j.ncat, st, tr)) != cudaSuccess) return e;
    Tables tb = tables_of(c);
    tb.stab = b->stab_f;
    return launch_forward(N, b->grid, b->spec, b->scal, tb, st, tr, j.ncat);
}

// Windows w0 .. of order index o, bins b0 .. b0+S-1, catalogues c0 .. c0+C-1.
cudaError_t batch_enqueue_window_block(hermes_ctx* c, const BatchJob& j, int o, int b0, int S, int c0, int C,
                                       cudaStream_t st, const Tracer& tr) {
    BatchState* b = c->batch;
    const int N = c->N, nb = c->n_bins, H = N / 2;
    const int ell = j.ells[o];
    const size_t n3 = (size_t)N * N * N;
    const int nwin = (int)j.ells.size() * nb;
    WinBatch wb;
    wb.S = S;
    wb.tab = c->rad + (size_t)ell * c->Q * c->nbp + b0;
    wb.nbp = c->nbp;
    wb.ell = ell;
    wb.scale = (float)((2 * ell + 1) * (((ell / 2) & 1) ? -1 : 1));
    const Tables tb = tables_of(c);
    const int zb = (C == 1) ? inv_z_blocks(N) : inv_z_blocks_plain(N);
    double* dd_part = b->part;
    cudaError_t e = launch_inverse_xi(N, b->spec + (size_t)c0 * N * N * H, b->work, b->grid + (size_t)c0 * n3, wb, tb,
                                      dd_part, c->err, st, tr, C);
    if (e != cudaSuccess) return e;
    double* dd = b->res;
    const size_t at = (size_t)c0 * nwin + (size_t)o * nb + b0;
    return launch_reduce_rows_strided(dd_part, C * S, zb, S, dd + at, nwin, st, tr);
}

cudaError_t batch_enqueue_windows(hermes_ctx* c, const BatchJob& j, cudaStream_t st, const Tracer& tr) {
    BatchState* b = c->batch;
    const int nb = c->n_bins;
    const int nwin = (int)j.ells.size() * nb;
    const int S = j.plan.S, C = j.plan.C;
    cudaError_t e;
    // self-pair terms, catalogue by catalogue (the histogram lives in the partials buffer)
    for (int k = 0; k < j.ncat; ++k) {
        Tables tb = tables_of(c);
        tb.stab = b->stab_f + (size_t)k * STAB_STRIDE;
        if ((e = enqueue_selfpair_terms(c, tb, j.ells.data(), (int)j.ells.size(), b->part,
                                        b->res + (size_t)j.ncat * nwin + (size_t)k * nwin, st, tr)) != cudaSuccess)
            return e;
    }
    for (int o = 0; o < (int)j.ells.size(); ++o)
        for (int b0 = 0; b0 < nb; b0 += S)
            for (int c0 = 0; c0 < j.ncat; c0 += C)
                if ((e = batch_enqueue_window_block(c, j, o, b0, std::min(S, nb - b0), c0, std::min(C, j.ncat - c0),
                                                    st, tr)) != cudaSuccess)
                    return e;
    double* dd = b->res;
    double* sn = b->res + (size_t)j.ncat * nwin;
    return launch_xi_batch_finish(dd, sn, b->scal, j.ncat, nwin, c->N, b->res + 2 * (size_t)j.ncat * nwin, st, tr);
}

}  // namespace

namespace {

// Candidate plans, timed on the live spectra with CUDA events: first S (windows
// per launch) at a middle C, then C (catalogues per launch) at the best S.  A
// candidate costs ms per catalogue-window; the cheapest wins.  Work-buffer size
// bounds both.
int batch_autotune(hermes_ctx* c, BatchJob& j, cudaStream_t st) {
    BatchState* b = c->batch;
    const int N = c->N, nb = c->n_bins;
    const size_t win_bytes = (size_t)N * N * (N / 2) * sizeof(float2);
    const size_t limit = batch_work_limit(c);
    const int nb4 = (nb + 3) & ~3;
    std::vector<int> Ss, Cs;
    for (int S : {4, 8, 16, 32})
        if (S <= std::max(4, nb4)) Ss.push_back(S);
    for (int C = 1; C <= j.ncat; C *= 2) Cs.push_back(C);
    if (Cs.back() != j.ncat) Cs.push_back(j.ncat);
    auto fits = [&](int S, int C) { return (size_t)S * C * win_bytes <= limit; };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "tuning event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, cudaErrorMemoryAllocation, "tuning event");
    }
    const Tracer quiet{c, count_only_mark};
    b->tune_ms.clear();
    auto trial = [&](int S, int C, double& ms_out) -> cudaError_t {
        const int Se = std::min(S, nb), Ce = std::min(C, j.ncat);
        cudaError_t e = batch_grow(c, j, Se, Ce);
        if (e != cudaSuccess) return e;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {  // first repetition warms up
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
            if ((e = batch_enqueue_window_block(c, j, 0, 0, Se, 0, Ce, st, quiet)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
            if (rep > 0) best = std::min(best, ms);
        }
        ms_out = best / ((double)Se * Ce);
        b->tune_ms.insert(b->tune_ms.end(), {(double)S, (double)C, ms_out});
        return cudaSuccess;
    };
    int rc = HERMES_OK;
    BatchPlan best;
    double best_ms = 1e300;
    const int C_mid = std::min(j.ncat, 8);
    for (int S : Ss) {
        if (!fits(S, C_mid)) continue;
        double ms;
        cudaError_t e = trial(S, C_mid, ms);
        if (e != cudaSuccess) {
            rc = cuda_fail(c, e, "autotune (windows per launch)");
            break;
        }
        if (ms < best_ms) best_ms = ms, best.S = S, best.C = C_mid;
    }
    if (rc == HERMES_OK && best.S == 0) rc = fail(c, HERMES_ERR_NOMEM, "no batch plan fits the free device memory");
    if (rc == HERMES_OK) {
        const int S = best.S;
        for (int C : Cs) {
            if (C == C_mid || !fits(S, C)) continue;
            double ms;
            cudaError_t e = trial(S, C, ms);
            if (e != cudaSuccess) {
                rc = cuda_fail(c, e, "autotune (catalogues per launch)");
                break;
            }
            if (ms < best_ms) best_ms = ms, best.C = C;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == HERMES_OK) j.plan = best;
    return rc;
}

std::vector<int64_t> batch_key(const hermes_ctx* c, const BatchJob& j) {
    const BatchState* b = c->batch;
    std::vector<int64_t> k = {c->N, c->p, j.ncat, j.n_total, j.has_w, j.wrap, c->n_bins, j.plan.S, j.plan.C,
                              (int64_t)(intptr_t)c->rad, (int64_t)(intptr_t)b->pos, (int64_t)(intptr_t)b->grid,
                              (int64_t)(intptr_t)b->part, (int64_t)(intptr_t)b->res, (int64_t)(intptr_t)b->work,
                              (int64_t)(intptr_t)c->stream};
    for (int e : j.ells) k.push_back(e);
    return k;
}

void counting_mark(void* vc, int, int phase, cudaStream_t) {
    if (phase == 0) ++((BatchState*)vc)->graph_kernels;
}

}  // namespace

extern "C" int hermes_batch_set_plan(hermes_ctx* c, int S, int C) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if ((S == 0) != (C == 0)) return fail(c, HERMES_ERR_ARG, "S and C are both 0 (autotune) or both positive");
    if (S < 0 || C < 0 || (S && (S % 4 || S > MAX_BATCH)) || C > MAX_CATALOGUES)
        return fail(c, HERMES_ERR_ARG, "S must be a multiple of 4 in 4..%d and C in 1..%d", MAX_BATCH,
                    MAX_CATALOGUES);
    if (!c->batch) c->batch = new BatchState;
    c->batch->forced = BatchPlan{S, C};
    return HERMES_OK;
}

extern "C" int hermes_batch_info(hermes_ctx* c, int* S, int* C, int64_t* graph_kernels, int64_t* graph_replays,
                                 double* tune, int tune_cap, int* n_tune) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    const BatchState* b = c->batch;
    if (S) *S = b ? b->last.S : 0;
    if (C) *C = b ? b->last.C : 0;
    if (graph_kernels) *graph_kernels = b ? b->graph_kernels : 0;
    if (graph_replays) *graph_replays = b ? b->graph_launches : 0;
    const int n = b ? (int)(b->tune_ms.size() / 3) : 0;
    if (n_tune) *n_tune = n;
    if (tune)
        for (int i = 0; i < std::min(n, tune_cap) * 3; ++i) tune[i] = b->tune_ms[i];
    return HERMES_OK;
}

extern "C" int hermes_xi_multipoles_batch(hermes_ctx* c, const float* pos, const float* w, const int64_t* offsets,
                                          int n_cat, const int* ells, int n_ells, unsigned flags, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!pos || !offsets || !ells || !out) return fail(c, HERMES_ERR_ARG, "pos/offsets/ells/out is NULL");
    if (n_cat < 1 || n_cat > MAX_CATALOGUES)
        return fail(c, HERMES_ERR_ARG, "n_cat = %d outside 1..%d", n_cat, MAX_CATALOGUES);
    if (n_ells < 1 || n_ells > 8) return fail(c, HERMES_ERR_ARG, "n_ells = %d outside 1..8", n_ells);
    if (flags & ~(HERMES_DEVICE_PTR | HERMES_WRAP | HERMES_EAGER))
        return fail(c, HERMES_ERR_ARG, "unknown flags 0x%x", flags);
    if (c->n_bins < 1) return fail(c, HERMES_ERR_STATE, "no bins: call hermes_window_shells first");
    if (offsets[0] != 0) return fail(c, HERMES_ERR_ARG, "offsets[0] = %lld, must be 0", (long long)offsets[0]);
    for (int k = 0; k < n_cat; ++k)
        if (offsets[k + 1] <= offsets[k])
            return fail(c, HERMES_ERR_ARG, "catalogue %d is empty or offsets decrease (the density contrast of an "
                                           "empty catalogue is undefined)", k);
    BatchJob j;
    j.ncat = n_cat;
    j.n_total = offsets[n_cat];
    j.has_w = w != nullptr;
    j.wrap = (flags & HERMES_WRAP) != 0;
    for (int a = 0; a < n_ells; ++a) {
        if (ells[a] < 0 || ells[a] > c->l_max)
            return fail(c, HERMES_ERR_ARG, "l = %d outside 0..l_max = %d", ells[a], c->l_max);
        if (ells[a] & 1) return fail(c, HERMES_ERR_ARG, "odd l = %d vanishes for an auto-correlation", ells[a]);
        j.ells.push_back(ells[a]);
    }
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    if (flags & HERMES_DEVICE_PTR) {
        int r = check_device_ptr(c, pos, "pos");
        if (r) return r;
        if (w && (r = check_device_ptr(c, w, "w"))) return r;
    }
    if (!c->batch) c->batch = new BatchState;
    BatchState* b = c->batch;
    cudaStream_t st = c->stream;
    const int nb = c->n_bins;
    // plan: forced, cached for this shape, or tuned below
    j.plan = b->forced;
    const std::vector<int64_t> pkey = {c->device, c->N, c->p, n_cat, nb, n_ells};
    bool tune = false;
    if (j.plan.S == 0) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(pkey);
        if (it != g_plans.end()) j.plan = it->second;
        else tune = true;
    }
    const int S0 = tune ? 4 : std::min(j.plan.S, nb), C0 = tune ? 1 : std::min(j.plan.C, n_cat);
    CK(batch_grow(c, j, S0, C0), "batch buffers");
    // inputs go to fixed device buffers, so a captured graph stays valid across calls
    const cudaMemcpyKind kind = (flags & HERMES_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(b->pos, pos, (size_t)j.n_total * 3 * sizeof(float), kind, st), "copy positions");
    if (w) CK(cudaMemcpyAsync(b->w, w, (size_t)j.n_total * sizeof(float), kind, st), "copy weights");
    CK(cudaMemcpyAsync(b->offs, offsets, (size_t)(n_cat + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st),
       "copy offsets");
    if (tune) {
        CK(batch_enqueue_assign(c, j, st, c->tracer), "batch fields for tuning");
        int r = batch_autotune(c, j, st);
        if (r) return r;
        {
            std::lock_guard<std::mutex> lk(g_plan_mu);
            g_plans[pkey] = j.plan;
        }
        CK(batch_grow(c, j, std::min(j.plan.S, nb), std::min(j.plan.C, n_cat)), "batch buffers");
    }
    const bool graphable =
        !(flags & HERMES_EAGER) && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    if (graphable) {
        const std::vector<int64_t> key = batch_key(c, j);
        if (!b->exec || key != b->key) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = nullptr;
            b->key.clear();
            b->graph_kernels = 0;
            const Tracer counting{b, counting_mark};
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin graph capture");
            cudaError_t e = batch_enqueue_assign(c, j, st, counting);
            if (e == cudaSuccess) e = batch_enqueue_windows(c, j, st, counting);
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(c, e != cudaSuccess ? e : e2, "capture of the batch graph");
            }
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                b->exec = nullptr;
                return cuda_fail(c, e, "instantiate the batch graph");
            }
            b->graph = graph;
            b->key = key;
        }
        c->tracer(K_BATCH_GRAPH, 0, st);
        CK(cudaGraphLaunch(b->exec, st), "launch the batch graph");
        c->tracer(K_BATCH_GRAPH, 1, st);
        c->launches += b->graph_kernels - 1;  // the tracer counted the graph as one launch
        ++b->graph_launches;
    } else {
        CK(batch_enqueue_assign(c, j, st, c->tracer), "batch fields");
        CK(batch_enqueue_windows(c, j, st, c->tracer), "batch windows");
    }
    const size_t nwin = (size_t)n_ells * nb;
    const size_t nres = (size_t)n_cat * nwin, nsc = (size_t)n_cat * SCAL_STRIDE;
    CK(ensure_host(c, nres + nsc + 1) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, b->res + 2 * nres, nres * sizeof(double), cudaMemcpyDeviceToHost, st), "read xi");
    CK(cudaMemcpyAsync(c->host_buf + nres, b->scal, nsc * sizeof(double), cudaMemcpyDeviceToHost, st), "read sums");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + nres + nsc);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "batch");
    b->last = j.plan;
    if (*hflag & 1u)
        return fail(c, HERMES_ERR_RANGE, "a coordinate is outside [0, L] (u = x*N/L outside [0, N]) or a weight is "
                                         "not finite; use HERMES_WRAP to wrap");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
    for (int k = 0; k < n_cat; ++k) {
        const double sw = c->host_buf[nres + (size_t)k * SCAL_STRIDE];
        if (!(sw > 0.0) || !std::isfinite(sw))
            return fail(c, HERMES_ERR_RANGE, "catalogue %d: sum of weights is %g; it must be positive", k, sw);
    }
    std::memcpy(out, c->host_buf, nres * sizeof(double));
    return HERMES_OK;
}

// ---------------------------------------------------------------------------
// Device-memory accounting (used by the request server's admission control).

extern "C" int64_t hermes_device_bytes(const hermes_ctx* c) {
    if (!c) return -1;
    const size_t N = (size_t)c->N, n3 = N * N * N;
    size_t b = n3 * sizeof(float) + N * N * (N / 2) * sizeof(float2);  // grid, spectrum
    b += TW_ENTRIES * sizeof(float2) + N * sizeof(float) + 8 * sizeof(double) + 512 * (sizeof(double) + sizeof(float));
    b += c->work_bytes + c->zfields_bytes + (c->part_cap + c->red_cap) * sizeof(double);
    b += c->stage_cap * 4 * sizeof(float);
    b += c->ts_pts_cap * 2 * sizeof(int) + c->ts_regions_cap * sizeof(float);
    if (c->ts_tiles) b += (3 * (size_t)scatter_tiled_tiles(c->N) + 1) * sizeof(int);
    if (c->rad) b += (size_t)c->nbp * (c->l_max + 1) * c->Q * sizeof(float);
    if (c->cyl_perp) b += ((size_t)c->cyl_nbp * c->cyl_Q + (size_t)c->cyl_npar * (N / 2)) * sizeof(float);
    if (c->rgrid) b += n3 * sizeof(float) + N * N * (N / 2) * sizeof(float2);
    if (c->batch) {
        const BatchState* s = c->batch;
        b += s->pts_cap * 4 * sizeof(float) + (size_t)s->cat_cap * (n3 * sizeof(float) + N * N * (N / 2) * sizeof(float2));
        b += s->work_bytes + (s->part_cap + s->res_cap) * sizeof(double);
    }
    return (int64_t)b;
}

extern "C" int64_t hermes_estimate_bytes(int N, int stat, int n_bins, int l_max, int64_t n_points, int host_inputs) {
    if (!valid_N(N) || n_bins < 1 || l_max < 0 || n_points < 0 || stat < 0 || stat > 2) return -1;
    const size_t n = (size_t)N, n3 = n * n * n;
    size_t b = n3 * sizeof(float) + n * n * (n / 2) * sizeof(float2);
    b += TW_ENTRIES * sizeof(float2) + n * sizeof(float) + 8 * sizeof(double) + 512 * (sizeof(double) + sizeof(float));
    const size_t nbp = (size_t)((n_bins + 3) & ~3);
    b += nbp * (size_t)(l_max + 1) * (size_t)table_len(N) * sizeof(float);
    if (host_inputs) b += (size_t)n_points * 4 * sizeof(float);
    // tiled scatter: per-point tile and permutation, per-tile tables, deposit regions (order p <= 8)
    b += (size_t)n_points * 2 * sizeof(int) + (3 * (size_t)scatter_tiled_tiles(N) + 1) * sizeof(int) +
         scatter_tiled_region_floats(N, 8) * sizeof(float);
    b += (size_t)std::max(2, 512) * 592 * sizeof(double) + 1024 * sizeof(double);  // assign partials
    if (stat == 2) {
        const size_t nblk = (size_t)(n_bins + 7) / 8, nruns = n_bins <= 16 ? 1 : nblk * (nblk + 1) / 2;
        b += (size_t)std::min(n_bins, 16) * n3 * sizeof(float2) + (size_t)256 * zeta_z_blocks(N) * sizeof(double);
        b += (size_t)256 * (l_max + 1) * (l_max + 2) / 2 * nruns * sizeof(double);
    } else {
        const size_t S = xi_window_S(N, n_bins);
        b += S * n * n * (n / 2) * sizeof(float2);
        b += S * ((size_t)inv_x_blocks(N) + (size_t)std::max(inv_z_blocks(N), inv_z_blocks_plain(N))) * sizeof(double);
        b += (size_t)2 * (l_max + 1) * n_bins * sizeof(double);
    }
    return (int64_t)b;
}

// ---------------------------------------------------------------------------
// Axisymmetric windows: xi(r_perp, r_par) with finite transverse annuli and
// line-of-sight slab pairs (Sec. 3.4.4; Table A1 rows (f)-(i) as limits).

namespace {

// Area average of J_0(k rho) over a <= rho < b: [b J_1(kb) - a J_1(ka)] / (k (b^2 - a^2) / 2),
// from int_0^r rho J_0(k rho) d rho = r J_1(k r) / k; 1 at k = 0.
double annulus_j0(double k, double a, double b) {
    if (k == 0.0) return 1.0;
    const double jb = b * ::j1(k * b);
    const double ja = a > 0.0 ? a * ::j1(k * a) : 0.0;
    return (jb - ja) / (k * 0.5 * (b * b - a * a));
}

// Average of cos(k z) over a <= |z| < b: [sin(kb) - sin(ka)] / (k (b - a)); 1 at k = 0.
double slab_cos(double k, double a, double b) {
    if (k == 0.0) return 1.0;
    return (std::sin(k * b) - std::sin(k * a)) / (k * (b - a));
}

}  // namespace

extern "C" int hermes_window_cylinders(hermes_ctx* c, const double* perp_edges, int n_perp_edges,
                                       const double* par_edges, int n_par_edges, double sigma_perp) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!perp_edges || !par_edges) return fail(c, HERMES_ERR_ARG, "edges are NULL");
    if (n_perp_edges < 2 || n_perp_edges > 4097 || n_par_edges < 2 || n_par_edges > 4097)
        return fail(c, HERMES_ERR_ARG, "need 2..4097 edges per axis (have %d transverse, %d line-of-sight)",
                    n_perp_edges, n_par_edges);
    if (!std::isfinite(sigma_perp) || sigma_perp < 0.0)
        return fail(c, HERMES_ERR_RANGE, "sigma_perp = %g must be finite and >= 0", sigma_perp);
    for (const auto& ax : {std::make_pair(perp_edges, n_perp_edges), std::make_pair(par_edges, n_par_edges)}) {
        for (int e = 0; e < ax.second; ++e) {
            if (!std::isfinite(ax.first[e]) || ax.first[e] < 0.0)
                return fail(c, HERMES_ERR_RANGE, "edge %d = %g is negative or not finite", e, ax.first[e]);
            if (e > 0 && !(ax.first[e] > ax.first[e - 1]))
                return fail(c, HERMES_ERR_RANGE, "edges must increase strictly (index %d)", e);
        }
        if (ax.first[ax.second - 1] > 0.5 * c->L)
            return fail(c, HERMES_ERR_RANGE, "largest edge %g exceeds L/2 = %g", ax.first[ax.second - 1], 0.5 * c->L);
    }
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const int N = c->N, H = N / 2;
    const int np = n_perp_edges - 1, nz = n_par_edges - 1;
    const int nbp = (np + 3) & ~3;
    const int64_t Qp = 2 * (int64_t)(H - 1) * (H - 1) + 1;  // q_perp = n_x^2 + n_y^2 off the Nyquist planes
    const double kf = 2.0 * M_PI / c->L;
    std::vector<float> perp, par;
    try {
        perp.assign((size_t)Qp * nbp, 0.0f);
        par.assign((size_t)nz * H, 0.0f);
    } catch (...) {
        return fail(c, HERMES_ERR_NOMEM, "host tables");
    }
    // transverse table by threads over q_perp (J_1 at every edge once per q)
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned w = 0; w < nt; ++w)
        th.emplace_back([&, w] {
            std::vector<double> rj(n_perp_edges);
            for (int64_t q = w; q < Qp; q += nt) {
                const double k = kf * std::sqrt((double)q);
                const double gs = std::exp(-0.5 * k * k * sigma_perp * sigma_perp);
                for (int i = 0; i < np; ++i)
                    perp[(size_t)q * nbp + i] = (float)(annulus_j0(k, perp_edges[i], perp_edges[i + 1]) * gs);
            }
        });
    for (auto& t : th) t.join();
    for (int j = 0; j < nz; ++j)
        for (int a = 0; a < H; ++a) par[(size_t)j * H + a] = (float)slab_cos(kf * a, par_edges[j], par_edges[j + 1]);
    cudaStreamSynchronize(c->stream);
    dev_free(c->cyl_perp);
    dev_free(c->cyl_par);
    c->cyl_perp = nullptr;
    c->cyl_par = nullptr;
    c->cyl_nperp = c->cyl_npar = 0;
    CK(dev_malloc((void**)&c->cyl_perp, perp.size() * sizeof(float)), "transverse table");
    CK(dev_malloc((void**)&c->cyl_par, par.size() * sizeof(float)), "line-of-sight table");
    CK(upload(c->cyl_perp, perp.data(), perp.size() * sizeof(float), c->stream), "upload tables");
    CK(upload(c->cyl_par, par.data(), par.size() * sizeof(float), c->stream), "upload tables");
    c->cyl_nperp = np;
    c->cyl_npar = nz;
    c->cyl_nbp = nbp;
    c->cyl_Q = Qp;
    c->cyl_ring = false;
    return HERMES_OK;
}

extern "C" int hermes_window_rings(hermes_ctx* c, const double* R, const double* Hz, const double* dRs,
                                   const double* dHs, int n, double sigma_perp) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!R || !Hz) return fail(c, HERMES_ERR_ARG, "R or H is NULL");
    if (n < 1 || n > 4096) return fail(c, HERMES_ERR_ARG, "need 1..4096 ring windows (have %d)", n);
    if (!std::isfinite(sigma_perp) || sigma_perp < 0.0)
        return fail(c, HERMES_ERR_RANGE, "sigma_perp = %g must be finite and >= 0", sigma_perp);
    for (int w = 0; w < n; ++w) {
        const double dR = dRs ? dRs[w] : 0.0, dH = dHs ? dHs[w] : 0.0;
        if (!std::isfinite(R[w]) || !std::isfinite(Hz[w]) || R[w] < 0.0 || Hz[w] < 0.0)
            return fail(c, HERMES_ERR_RANGE, "ring %d: R = %g, H = %g must be finite and >= 0", w, R[w], Hz[w]);
        if (!std::isfinite(dR) || !std::isfinite(dH) || dR < 0.0 || dH < 0.0)
            return fail(c, HERMES_ERR_RANGE, "ring %d: widths dR = %g, dH = %g must be finite and >= 0", w, dR, dH);
        if (R[w] + 0.5 * dR > 0.5 * c->L || Hz[w] + 0.5 * dH > 0.5 * c->L)
            return fail(c, HERMES_ERR_RANGE, "ring %d reaches beyond L/2 = %g", w, 0.5 * c->L);
    }
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    const int N = c->N, H = N / 2;
    const int nbp = (n + 3) & ~3;
    const int64_t Qp = 2 * (int64_t)(H - 1) * (H - 1) + 1;
    const double kf = 2.0 * M_PI / c->L;
    std::vector<float> perp, par;
    try {
        perp.assign((size_t)Qp * nbp, 0.0f);
        par.assign((size_t)n * H, 0.0f);
    } catch (...) {
        return fail(c, HERMES_ERR_NOMEM, "host tables");
    }
    // Sec. 3.4.4: the thin double ring J_0(k_perp R) cos(k_par H); finite widths give the
    // area average of J_0 over the transverse bin R +- dR/2 and the average of cos(k_par z)
    // over the line-of-sight bin H +- dH/2 (sin(k dH/2)/(k dH/2) cos(k H)), each bin
    // clipped at 0 where it would reach below (the separations the pairs actually cover)
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int64_t q = t; q < Qp; q += nt) {
                const double k = kf * std::sqrt((double)q);
                const double gs = std::exp(-0.5 * k * k * sigma_perp * sigma_perp);
                for (int w = 0; w < n; ++w) {
                    const double dR = dRs ? dRs[w] : 0.0;
                    const double v = dR > 0.0 ? annulus_j0(k, std::max(0.0, R[w] - 0.5 * dR), R[w] + 0.5 * dR)
                                              : ::j0(k * R[w]);
                    perp[(size_t)q * nbp + w] = (float)(v * gs);
                }
            }
        });
    for (auto& t : th) t.join();
    for (int w = 0; w < n; ++w)
        for (int a = 0; a < H; ++a) {
            const double k = kf * a, dH = dHs ? dHs[w] : 0.0;
            par[(size_t)w * H + a] =
                (float)(dH > 0.0 ? slab_cos(k, std::max(0.0, Hz[w] - 0.5 * dH), Hz[w] + 0.5 * dH)
                                 : std::cos(k * Hz[w]));
        }
    cudaStreamSynchronize(c->stream);
    dev_free(c->cyl_perp);
    dev_free(c->cyl_par);
    c->cyl_perp = nullptr;
    c->cyl_par = nullptr;
    c->cyl_nperp = c->cyl_npar = 0;
    CK(dev_malloc((void**)&c->cyl_perp, perp.size() * sizeof(float)), "ring transverse table");
    CK(dev_malloc((void**)&c->cyl_par, par.size() * sizeof(float)), "ring line-of-sight table");
    CK(upload(c->cyl_perp, perp.data(), perp.size() * sizeof(float), c->stream), "upload tables");
    CK(upload(c->cyl_par, par.data(), par.size() * sizeof(float), c->stream), "upload tables");
    c->cyl_nperp = n;
    c->cyl_npar = n;
    c->cyl_nbp = nbp;
    c->cyl_Q = Qp;
    c->cyl_ring = true;
    return HERMES_OK;
}

namespace {
int check_cyl(hermes_ctx* c, double* out, bool ring = false) {
    if (!out) return fail(c, HERMES_ERR_ARG, "out is NULL");
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->cyl_nperp < 1 || c->cyl_ring != ring)
        return fail(c, HERMES_ERR_STATE, ring ? "no ring windows: call hermes_window_rings first"
                                              : "no cylindrical bins: call hermes_window_cylinders first");
    return HERMES_OK;
}
}  // namespace

extern "C" int hermes_xi_cylinders(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (int r = check_cyl(c, out)) return r;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, H = N / 2, np = c->cyl_nperp, nz = c->cyl_npar;
    const int nwin = np * nz;
    const size_t win_bytes = (size_t)N * N * H * sizeof(float2);
    const int S = (int)xi_window_S(N, np);
    CK(grow(c->work, c->work_bytes, (size_t)S * win_bytes), "window work buffer");
    const int zb = inv_z_blocks(N);
    CK(grow_doubles(c->part, c->part_cap, std::max((size_t)S * zb, (size_t)std::min(nz, 8) * c->cyl_Q)), "partials");
    CK(grow_doubles(c->red, c->red_cap, (size_t)3 * nwin), "reduction buffer");  // dd, sn, RR
    const Tables tb = tables_of(c);
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    std::vector<int> js(nz);
    for (int j = 0; j < nz; ++j) js[j] = j;
    CK(enqueue_hist_terms(c, tb, nullptr, js.data(), nz, 1, 1, c->part, c->red + nwin, st, c->tracer),
       "self-pair terms");
    for (int j = 0; j < nz; ++j)
        for (int b0 = 0; b0 < np; b0 += S) {
            WinBatch wb;
            wb.S = std::min(S, np - b0);
            wb.tab = c->cyl_perp + b0;
            wb.nbp = c->cyl_nbp;
            wb.ell = 0;
            wb.scale = 1.0f;
            wb.cyl = 1;
            wb.par = c->cyl_par + (size_t)j * H;
            CK(launch_inverse_xi(N, c->spec, c->work, c->grid, wb, tb, c->part, c->err, st, c->tracer),
               "inverse passes");
            CK(launch_reduce_rows(c->part, wb.S, zb, c->red + (size_t)j * np + b0, st, c->tracer),
               "reduce contractions");
        }
    const int nrr = c->have_randoms ? nwin : 0;
    if (nrr) CK(enqueue_rr_terms(c, js.data(), nz, 1, c->part, c->red + 2 * nwin, st, c->tracer), "random pairs");
    CK(ensure_host(c, (size_t)2 * nwin + nrr + 1) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation,
       "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(2 * nwin + nrr) * sizeof(double), cudaMemcpyDeviceToHost, st),
       "read xi");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + (size_t)2 * nwin + nrr);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "xi(r_perp, r_par)");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
    const double n3 = (double)N * N * N, n6 = n3 * n3, eb = c->sum_w / n3;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int w = 0; w < nwin; ++w)
        out[w] = (c->host_buf[w] / n6 - c->host_buf[nwin + w] / (eb * eb)) /
                 (nrr ? c->host_buf[2 * nwin + w] * rr_scale : 1.0);
    return HERMES_OK;
}

extern "C" int hermes_xi_cylinders_kspace(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (int r = check_cyl(c, out)) return r;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int np = c->cyl_nperp, nz = c->cyl_npar, nwin = np * nz;
    CK(grow_doubles(c->part, c->part_cap, (size_t)std::min(nz, 8) * c->cyl_Q), "histogram");
    CK(grow_doubles(c->red, c->red_cap, (size_t)2 * nwin), "reduction buffer");  // xi numerators, RR
    std::vector<int> js(nz);
    for (int j = 0; j < nz; ++j) js[j] = j;
    CK(enqueue_hist_terms(c, tables_of(c), c->scal, js.data(), nz, 1, 0, c->part, c->red, st, c->tracer),
       "k-space histogram");
    const int nrr = c->have_randoms ? nwin : 0;
    if (nrr) CK(enqueue_rr_terms(c, js.data(), nz, 1, c->part, c->red + nwin, st, c->tracer), "random pairs");
    CK(ensure_host(c, (size_t)nwin + nrr) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(nwin + nrr) * sizeof(double), cudaMemcpyDeviceToHost, st),
       "read xi");
    CK(cudaStreamSynchronize(st), "xi(r_perp, r_par) (k-space)");
    const double n3 = (double)c->N * c->N * c->N;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int w = 0; w < nwin; ++w) out[w] = c->host_buf[w] / (nrr ? c->host_buf[nwin + w] * rr_scale : 1.0);
    return HERMES_OK;
}

extern "C" int hermes_xi_rings(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (int r = check_cyl(c, out, true)) return r;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, H = N / 2, nwin = c->cyl_nperp;
    const size_t win_bytes = (size_t)N * N * H * sizeof(float2);
    const int S = (int)xi_window_S(N, nwin);
    CK(grow(c->work, c->work_bytes, (size_t)S * win_bytes), "window work buffer");
    const int zb = inv_z_blocks(N);
    CK(grow_doubles(c->part, c->part_cap, std::max((size_t)S * zb, (size_t)std::min(nwin, 8) * c->cyl_Q)),
       "partials");
    CK(grow_doubles(c->red, c->red_cap, (size_t)3 * nwin), "reduction buffer");  // dd, sn, RR
    const Tables tb = tables_of(c);
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    std::vector<int> ws(nwin);
    for (int w = 0; w < nwin; ++w) ws[w] = w;
    CK(enqueue_hist_terms(c, tb, nullptr, ws.data(), nwin, 1, 1, c->part, c->red + nwin, st, c->tracer),
       "self-pair terms");
    for (int w0 = 0; w0 < nwin; w0 += S) {
        WinBatch wb;
        wb.S = std::min(S, nwin - w0);
        wb.tab = c->cyl_perp + w0;
        wb.nbp = c->cyl_nbp;
        wb.ell = 0;
        wb.scale = 1.0f;
        wb.cyl = 1;
        wb.par = c->cyl_par + (size_t)w0 * H;
        wb.par_stride = H;
        CK(launch_inverse_xi(N, c->spec, c->work, c->grid, wb, tb, c->part, c->err, st, c->tracer), "inverse passes");
        CK(launch_reduce_rows(c->part, wb.S, zb, c->red + w0, st, c->tracer), "reduce contractions");
    }
    const int nrr = c->have_randoms ? nwin : 0;
    if (nrr) CK(enqueue_rr_terms(c, ws.data(), nwin, 1, c->part, c->red + 2 * nwin, st, c->tracer), "random pairs");
    CK(ensure_host(c, (size_t)2 * nwin + nrr + 1) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation,
       "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(2 * nwin + nrr) * sizeof(double), cudaMemcpyDeviceToHost, st),
       "read xi");
    unsigned* hflag = reinterpret_cast<unsigned*>(c->host_buf + (size_t)2 * nwin + nrr);
    CK(cudaMemcpyAsync(hflag, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "xi over ring windows");
    if (*hflag & 4u) return fail(c, HERMES_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
    const double n3 = (double)N * N * N, n6 = n3 * n3, eb = c->sum_w / n3;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int w = 0; w < nwin; ++w)
        out[w] = (c->host_buf[w] / n6 - c->host_buf[nwin + w] / (eb * eb)) /
                 (nrr ? c->host_buf[2 * nwin + w] * rr_scale : 1.0);
    return HERMES_OK;
}

extern "C" int hermes_xi_rings_kspace(hermes_ctx* c, double* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (int r = check_cyl(c, out, true)) return r;
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int nwin = c->cyl_nperp;
    CK(grow_doubles(c->part, c->part_cap, (size_t)std::min(nwin, 8) * c->cyl_Q), "histogram");
    CK(grow_doubles(c->red, c->red_cap, (size_t)2 * nwin), "reduction buffer");  // xi numerators, RR
    std::vector<int> ws(nwin);
    for (int w = 0; w < nwin; ++w) ws[w] = w;
    CK(enqueue_hist_terms(c, tables_of(c), c->scal, ws.data(), nwin, 1, 0, c->part, c->red, st, c->tracer),
       "k-space histogram");
    const int nrr = c->have_randoms ? nwin : 0;
    if (nrr) CK(enqueue_rr_terms(c, ws.data(), nwin, 1, c->part, c->red + nwin, st, c->tracer), "random pairs");
    CK(ensure_host(c, (size_t)nwin + nrr) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, (size_t)(nwin + nrr) * sizeof(double), cudaMemcpyDeviceToHost, st),
       "read xi");
    CK(cudaStreamSynchronize(st), "xi over ring windows (k-space)");
    const double n3 = (double)c->N * c->N * c->N;
    const double rr_scale = nrr ? (n3 / c->sum_wr) * (n3 / c->sum_wr) : 0.0;
    for (int w = 0; w < nwin; ++w) out[w] = c->host_buf[w] / (nrr ? c->host_buf[nwin + w] * rr_scale : 1.0);
    return HERMES_OK;
}

// ---------------------------------------------------------------------------
// Explicit random catalogue (Landy-Szalay in the field language, Sec. 3.3).

extern "C" int hermes_assign_randoms(hermes_ctx* c, const float* pos, const float* w, int64_t n, unsigned flags) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!pos) return fail(c, HERMES_ERR_ARG, "pos is NULL");
    if (n < 1) return fail(c, HERMES_ERR_ARG, "empty random catalogue");
    if (flags & ~(HERMES_DEVICE_PTR | HERMES_WRAP)) return fail(c, HERMES_ERR_ARG, "unknown flags 0x%x", flags);
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, p = c->p, p3 = p * p * p;
    const size_t n3 = (size_t)N * N * N;
    const float* dpos = pos;
    const float* dw = w;
    if (flags & HERMES_DEVICE_PTR) {
        int r = check_device_ptr(c, pos, "pos");
        if (r) return r;
        if (w && (r = check_device_ptr(c, w, "w"))) return r;
    } else {
        if ((size_t)n > c->stage_cap) {
            dev_free(c->stage_pos);
            dev_free(c->stage_w);
            c->stage_pos = nullptr;
            c->stage_w = nullptr;
            c->stage_cap = 0;
            CK(dev_malloc((void**)&c->stage_pos, (size_t)n * 3 * sizeof(float)), "staging positions");
            CK(dev_malloc((void**)&c->stage_w, (size_t)n * sizeof(float)), "staging weights");
            c->stage_cap = (size_t)n;
        }
        CK(cudaMemcpyAsync(c->stage_pos, pos, (size_t)n * 3 * sizeof(float), cudaMemcpyDefault, st), "copy positions");
        if (w) CK(cudaMemcpyAsync(c->stage_w, w, (size_t)n * sizeof(float), cudaMemcpyDefault, st), "copy weights");
        dpos = c->stage_pos;
        dw = w ? c->stage_w : nullptr;
    }
    if (!c->rgrid) CK(dev_malloc((void**)&c->rgrid, n3 * sizeof(float)), "random field");
    if (!c->rspec) CK(dev_malloc((void**)&c->rspec, (size_t)N * N * (N / 2) * sizeof(float2)), "random spectrum");
    if (!c->rstab_d) CK(dev_malloc((void**)&c->rstab_d, 512 * sizeof(double)), "random self-pair table");
    if (!c->rstab_f) CK(dev_malloc((void**)&c->rstab_f, 512 * sizeof(float)), "random self-pair table");
    if (!c->rscal) {
        CK(dev_malloc((void**)&c->rscal, 8 * sizeof(double)), "random scalars");
        const double one[8] = {0, 0, 1, 0, 0, 0, 0, 0};
        CK(upload(c->rscal, one, sizeof(one), c->stream), "random scalars");
    }
    c->have_field = false;  // the data field must be rebuilt against the new randoms
    c->have_randoms = false;
    const int nblk = 592;
    CK(grow_doubles(c->part, c->part_cap, (size_t)std::max(2, p3) * nblk), "partials");
    CK(grow_doubles(c->red, c->red_cap, 1024), "reduction buffer");
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    const float s = (float)((double)N / c->L);
    CK(scatter_tiled(c, dpos, dw, n, c->rgrid, s, (flags & HERMES_WRAP) ? 1 : 0, st), "scatter randoms");
    CK(launch_weight_sums(dw, n, c->part, nblk, st, c->tracer), "weight sums");
    CK(launch_reduce_rows(c->part, 2, nblk, c->red, st, c->tracer), "reduce sums");
    CK(launch_selfpair(N, p, dpos, dw, n, s, c->part, nblk, st, c->tracer), "self-pair table");
    CK(launch_reduce_rows(c->part, p3, nblk, c->rstab_d, st, c->tracer), "reduce self-pair");
    // float copy of the table (the scalars land in scratch)
    CK(launch_finish_field(c->red, c->rstab_d, p3, c->rstab_f, N, c->red + 8, st, c->tracer), "random table");
    CK(launch_delta_to_spec(N, c->rgrid, c->rspec, nullptr, tables_of(c), st, c->tracer, 1), "random spectrum");
    CK(ensure_host(c, 4) == HERMES_OK ? cudaSuccess : cudaErrorMemoryAllocation, "host buffer");
    CK(cudaMemcpyAsync(c->host_buf, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "read sums");
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    CK(cudaStreamSynchronize(st), "assign randoms");
    if (herr) return fail(c, HERMES_ERR_RANGE, "a random coordinate is outside [0, L] or a weight is not finite");
    c->sum_wr = c->host_buf[0];
    if (!(c->sum_wr > 0.0) || !std::isfinite(c->sum_wr))
        return fail(c, HERMES_ERR_RANGE, "sum of random weights is %g; it must be positive", c->sum_wr);
    c->have_randoms = true;
    return HERMES_OK;
}

extern "C" int hermes_clear_randoms(hermes_ctx* c) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (c->have_randoms) c->have_field = false;  // the resident field is a difference field
    c->have_randoms = false;
    return HERMES_OK;
}

// ---------------------------------------------------------------------------
// Density-dependent marks (Sec. 3.3): smoothed density read at the particles.

extern "C" int hermes_density_marks(hermes_ctx* c, int window, double R, int kind, double a, double b,
                                    int remove_self, const float* pos, int64_t n, unsigned flags, float* out) {
    if (check_ctx(c)) return HERMES_ERR_ARG;
    if (!pos || !out || n < 1) return fail(c, HERMES_ERR_ARG, "pos/out NULL or n < 1");
    if (window != HERMES_SMOOTH_SPHERE && window != HERMES_SMOOTH_GAUSS)
        return fail(c, HERMES_ERR_ARG, "unknown smoothing window %d", window);
    if (kind < HERMES_MARK_DENSITY || kind > HERMES_MARK_INVERSE) return fail(c, HERMES_ERR_ARG, "unknown mark %d", kind);
    if (!(R > 0.0) || !std::isfinite(R) || R > 0.5 * c->L)
        return fail(c, HERMES_ERR_RANGE, "smoothing radius %g outside (0, L/2]", R);
    if (!std::isfinite(a) || !std::isfinite(b)) return fail(c, HERMES_ERR_ARG, "mark parameters must be finite");
    if (flags & ~(HERMES_DEVICE_PTR | HERMES_WRAP)) return fail(c, HERMES_ERR_ARG, "unknown flags 0x%x", flags);
    if (!c->have_field) return fail(c, HERMES_ERR_STATE, "no field: call hermes_assign first");
    if (c->have_randoms)
        return fail(c, HERMES_ERR_STATE, "the resident field is a difference field (explicit randoms); "
                                         "call hermes_clear_randoms and hermes_assign first");
    DeviceGuard g(c->device);
    AllocStream as_(c->stream);
    cudaStream_t st = c->stream;
    const int N = c->N, H = N / 2;
    const size_t n3 = (size_t)N * N * N;
    const float* dpos = pos;
    float* dout = out;
    if (flags & HERMES_DEVICE_PTR) {
        int r = check_device_ptr(c, pos, "pos");
        if (r) return r;
        if ((r = check_device_ptr(c, out, "out"))) return r;
    } else {
        if ((size_t)n > c->stage_cap) {
            dev_free(c->stage_pos);
            dev_free(c->stage_w);
            c->stage_pos = nullptr;
            c->stage_w = nullptr;
            c->stage_cap = 0;
            CK(dev_malloc((void**)&c->stage_pos, (size_t)n * 3 * sizeof(float)), "staging positions");
            CK(dev_malloc((void**)&c->stage_w, (size_t)n * sizeof(float)), "staging marks");
            c->stage_cap = (size_t)n;
        }
        CK(cudaMemcpyAsync(c->stage_pos, pos, (size_t)n * 3 * sizeof(float), cudaMemcpyDefault, st), "copy positions");
        dpos = c->stage_pos;
        dout = c->stage_w;
    }
    // one-bin table W^(k_q) for q = |n|^2 (Table A1 rows (b), (c)), float64 on the host
    const int64_t Q = table_len(N);
    std::vector<float> tab((size_t)Q * 4, 0.0f);
    const double kf = 2.0 * M_PI / c->L;
    for (int64_t q = 0; q < Q; ++q) {
        const double x = kf * std::sqrt((double)q) * R;
        double wv;
        if (window == HERMES_SMOOTH_GAUSS) wv = std::exp(-0.5 * x * x);
        else if (x < 1e-2) wv = 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
        else wv = 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
        tab[(size_t)q * 4] = (float)wv;
    }
    cudaStreamSynchronize(st);
    dev_free(c->smooth_tab);
    c->smooth_tab = nullptr;
    CK(dev_malloc((void**)&c->smooth_tab, tab.size() * sizeof(float)), "smoothing table");
    CK(upload(c->smooth_tab, tab.data(), tab.size() * sizeof(float), c->stream), "upload table");
    // work: one half spectrum, then the real smoothed field (N^3 floats) behind it
    const size_t spec_bytes = (size_t)N * N * H * sizeof(float2);
    CK(grow(c->work, c->work_bytes, spec_bytes + n3 * sizeof(float)), "work buffer");
    float* field = reinterpret_cast<float*>(reinterpret_cast<char*>(c->work) + spec_bytes);
    WinBatch wb;
    wb.tab = c->smooth_tab;
    wb.nbp = 4;
    wb.S = 1;
    wb.ell = 0;
    wb.scale = 1.0f;
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "clear flag");
    CK(launch_smooth_field(N, c->spec, c->work, field, wb, tables_of(c), st, c->tracer), "smoothing");
    // one object per window volume, in units of the mean density sum w / L^3
    const double vol = window == HERMES_SMOOTH_GAUSS ? std::pow(2.0 * M_PI, 1.5) * R * R * R : 4.0 * M_PI * R * R * R / 3.0;
    const double self = remove_self ? c->L * c->L * c->L / (vol * c->sum_w) : 0.0;
    const float s = (float)((double)N / c->L);
    CK(launch_gather_marks(N, c->p, dpos, n, field, s, (flags & HERMES_WRAP) ? 1 : 0, kind, (float)a, (float)b,
                           (float)self, dout, c->err, st, c->tracer),
       "gather");
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read flag");
    if (!(flags & HERMES_DEVICE_PTR))
        CK(cudaMemcpyAsync(out, dout, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st), "read marks");
    CK(cudaStreamSynchronize(st), "density marks");
    if (herr) return fail(c, HERMES_ERR_RANGE, "a coordinate is outside [0, L]; use HERMES_WRAP to wrap");
    return HERMES_OK;
}
