// B-spline scatter of a weighted point catalogue onto the periodic N^3 grid,
// Eq. (phi_projection): eps_l = sum_i w_i prod_d M_p(u_{i,d} - l_d), plus the
// float64 cell-sum reductions (sum w, sum w^2) and the self-pair overlap table
// S(a,b,c) = sum_i w_i^2 prod_d s(a_d; x_i) with s(d; x) = sum_l phi_l(x) phi_{l+d}(x).
//
// Node rule (bit-exact with the oracle): u = fl32(x * s), s = fl32(N/L);
// v = u (+0.5 in float32 for odd p); i = floor(v); t = v - i; the p supporting
// nodes are i - (p/2 - 1) + o (even p) or i - (p-1)/2 + o (odd p), o = 0..p-1,
// all taken modulo N; node o carries the uniform B-spline basis value b_o(t).
#include "kernels.h"
#include "common.cuh"

namespace hermes {

// Uniform B-spline basis values b_0..b_{P-1} at local parameter t in [0,1):
// b_o = M_P(distance from node o), via the Cox-de Boor recursion on integer knots.
template <int P>
__device__ __forceinline__ void bspline_basis(float t, float (&b)[P]) {
    b[0] = 1.0f;
#pragma unroll
    for (int d = 1; d < P; ++d) {
        const float inv_d = 1.0f / (float)d;
        b[d] = 0.0f;
#pragma unroll
        for (int j = d; j >= 0; --j) {
            float left = (j > 0) ? (t + (float)(d - j)) * b[j - 1] : 0.0f;
            float right = (j < d) ? ((float)(j + 1) - t) * b[j] : 0.0f;
            b[j] = (left + right) * inv_d;
        }
    }
}

// Returns false if the coordinate is outside the accepted range.
template <int P>
__device__ __forceinline__ bool node_rule(float x, float s, int N, int wrap, int& first, float (&b)[P]) {
    const float u = __fmul_rn(x, s);
    const bool ok = wrap ? (fabsf(u) < 4194304.0f) : (u >= 0.0f && u <= (float)N);
    if (!ok) return false;
    const float v = (P & 1) ? __fadd_rn(u, 0.5f) : u;
    const float fl = floorf(v);
    const float t = __fsub_rn(v, fl);
    const int i0 = (int)fl;
    first = (P & 1) ? i0 - (P - 1) / 2 : i0 - (P / 2 - 1);
    bspline_basis<P>(t, b);
    return true;
}

// Adds w*b[c] to row[(z0 + c) mod N], c = 0..P-1, with as few atomic
// operations as the alignment allows: the run of P contiguous cells is cut at
// 16- and 8-byte boundaries into float4 / float2 / float atomics (vector
// atomics: sm_90+, natural alignment; rows start 16-byte aligned as N >= 16).
// A is (z0 mod 4), known per instantiation, so every index is static.
template <int P, int A, int C>
__device__ __forceinline__ void add_aligned(float* p, float w, const float (&b)[P]) {
    if constexpr (C < P) {
        constexpr int al = (A + C) & 3;
        if constexpr (al == 0 && C + 4 <= P) {
            atomicAdd(reinterpret_cast<float4*>(p + C), make_float4(w * b[C], w * b[C + 1], w * b[C + 2], w * b[C + 3]));
            add_aligned<P, A, C + 4>(p, w, b);
        } else if constexpr ((al & 1) == 0 && C + 2 <= P) {
            atomicAdd(reinterpret_cast<float2*>(p + C), make_float2(w * b[C], w * b[C + 1]));
            add_aligned<P, A, C + 2>(p, w, b);
        } else {
            atomicAdd(p + C, w * b[C]);
            add_aligned<P, A, C + 1>(p, w, b);
        }
    }
}

template <int P>
__device__ __forceinline__ void add_run(float* row, int z0, int N, float w, const float (&b)[P]) {
    if (z0 + P > N) {  // the run wraps around the periodic edge: scalar atomics
#pragma unroll
        for (int c = 0; c < P; ++c) atomicAdd(row + ((z0 + c) & (N - 1)), w * b[c]);
        return;
    }
    float* p = row + z0;
    switch (z0 & 3) {
        case 0: add_aligned<P, 0, 0>(p, w, b); break;
        case 1: add_aligned<P, 1, 0>(p, w, b); break;
        case 2: add_aligned<P, 2, 0>(p, w, b); break;
        default: add_aligned<P, 3, 0>(p, w, b); break;
    }
}

// One point's p^3 contributions (err bit 1 on a rejected coordinate or weight).
template <int P>
__device__ __forceinline__ void scatter_point(float x, float y, float z, float wi, float* __restrict__ grid, float s,
                                              int N, int wrap, unsigned* __restrict__ err) {
    const int msk = N - 1;
    float bx[P], by[P], bz[P];
    int fx, fy, fz;
    bool ok = node_rule<P>(x, s, N, wrap, fx, bx) & node_rule<P>(y, s, N, wrap, fy, by) &
              node_rule<P>(z, s, N, wrap, fz, bz);
    if (!ok || !isfinite(wi)) {
        atomicOr(err, 1u);
        return;
    }
    const int z0 = fz & msk;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const int ix = (fx + a) & msk;
        const float wa = wi * bx[a];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const int iy = (fy + b) & msk;
            const float wab = wa * by[b];
            float* row = grid + ((size_t)ix * N + iy) * N;
            add_run<P>(row, z0, N, wab, bz);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_scatter(const float* __restrict__ pos, const float* __restrict__ w,
                                                 int64_t n, float* __restrict__ grid, float s, int N, int wrap,
                                                 unsigned* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = __ldg(pos + 3 * i), y = __ldg(pos + 3 * i + 1), z = __ldg(pos + 3 * i + 2);
        const float wi = w ? __ldg(w + i) : 1.0f;
        scatter_point<P>(x, y, z, wi, grid, s, N, wrap, err);
    }
}

// Batched scatter of catalogues c0 .. c1-1: catalogue c owns points
// [offs[c], offs[c+1]) of one concatenated array and grid c (N^3 floats,
// consecutive grids).  The point range is read from the device offsets, so one
// launch configuration serves any split of the points.  The grid stride runs
// over the whole range, so uneven catalogues share the GPU evenly; each point
// finds its catalogue by bisection over the offsets held in shared memory.
// The host launches groups of catalogues whose grids fit in L2 together, so the
// atomics resolve in L2 instead of DRAM.
template <int P>
__global__ void __launch_bounds__(256) k_scatter_batch(const float* __restrict__ pos, const float* __restrict__ w,
                                                       const int64_t* __restrict__ offs, int c0, int c1,
                                                       float* __restrict__ grid, float s, int N, int wrap,
                                                       unsigned* __restrict__ err) {
    __shared__ int64_t so[MAX_CATALOGUES + 1];
    const int ncat = c1 - c0;
    for (int c = threadIdx.x; c <= ncat; c += blockDim.x) so[c] = offs[c0 + c];
    __syncthreads();
    const size_t n3 = (size_t)N * N * N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    grid += (size_t)c0 * n3;
    for (int64_t i = so[0] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < so[ncat]; i += stride) {
        int lo = 0, hi = ncat;  // so[lo] <= i < so[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (so[mid] <= i) lo = mid;
            else hi = mid;
        }
        const float x = __ldg(pos + 3 * i), y = __ldg(pos + 3 * i + 1), z = __ldg(pos + 3 * i + 2);
        const float wi = w ? __ldg(w + i) : 1.0f;
        scatter_point<P>(x, y, z, wi, grid + (size_t)lo * n3, s, N, wrap, err);
    }
}

// Adjoint of the scatter: read a field at the points through the same basis, then
// apply the density mark (see launch_gather_marks).
template <int P>
__global__ void __launch_bounds__(256) k_gather_marks(const float* __restrict__ pos, int64_t n,
                                                      const float* __restrict__ field, float s, int N, int wrap,
                                                      int kind, float ma, float mb, float self,
                                                      float* __restrict__ out, unsigned* __restrict__ err) {
    const int msk = N - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float bx[P], by[P], bz[P];
        int fx, fy, fz;
        const bool ok = node_rule<P>(__ldg(pos + 3 * i), s, N, wrap, fx, bx) &
                        node_rule<P>(__ldg(pos + 3 * i + 1), s, N, wrap, fy, by) &
                        node_rule<P>(__ldg(pos + 3 * i + 2), s, N, wrap, fz, bz);
        if (!ok) {
            atomicOr(err, 1u);
            out[i] = 0.0f;
            continue;
        }
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const int ix = (fx + a) & msk;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const float* row = field + ((size_t)ix * N + ((fy + b) & msk)) * N;
                float r = 0.0f;
#pragma unroll
                for (int c = 0; c < P; ++c) r = fmaf(bz[c], __ldg(row + ((fz + c) & msk)), r);
                acc = fmaf(bx[a] * by[b], r, acc);
            }
        }
        const float rho = 1.0f + acc;
        const float r = fmaxf(rho - self, 0.0f);
        out[i] = kind == 0 ? rho : (kind == 1 ? powf(r + mb, ma) : powf((mb + 1.0f) / (mb + r), ma));
    }
}

// ---------------------------------------------------------------------------
// Tiled scatter: shared-memory privatisation of the B-spline deposit.
//   1. each point's tile is the tile of its first node (tiles of SB^3 cells, NT
//      per axis); points are counted per tile,
//   2. an exclusive scan of the counts gives each tile's range of a permutation,
//      filled by a second pass,
//   3. one block per tile deposits its points into a shared region of
//      RB^3 = (SB + P - 1)^3 cells (the tile and the P - 1 cells its points reach
//      beyond it) with shared-memory atomics and writes the region out,
//   4. every grid cell sums the (up to 2 per axis) regions that cover it, with a
//      plain store; the grid needs no clearing and sees no global atomics.
constexpr int SB = 16;

__device__ __forceinline__ int tile_of_first(int fx, int fy, int fz, int N, int NT) {
    const int msk = N - 1;
    return (((fx & msk) / SB) * NT + (fy & msk) / SB) * NT + (fz & msk) / SB;
}

template <int P>
__global__ void __launch_bounds__(256) k_tile_count(const float* __restrict__ pos, const float* __restrict__ w,
                                                    int64_t n, float s, int N, int wrap, int NT,
                                                    int* __restrict__ counts, int* __restrict__ tile_of,
                                                    unsigned* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float bx[P], by[P], bz[P];
        int fx, fy, fz;
        const bool ok = node_rule<P>(__ldg(pos + 3 * i), s, N, wrap, fx, bx) &
                        node_rule<P>(__ldg(pos + 3 * i + 1), s, N, wrap, fy, by) &
                        node_rule<P>(__ldg(pos + 3 * i + 2), s, N, wrap, fz, bz);
        const float wi = w ? __ldg(w + i) : 1.0f;
        if (!ok || !isfinite(wi)) {
            atomicOr(err, 1u);
            tile_of[i] = -1;
            continue;
        }
        const int t = tile_of_first(fx, fy, fz, N, NT);
        tile_of[i] = t;
        atomicAdd(counts + t, 1);
    }
}

// Exclusive scan of n counts by one block of 1024 threads; offs[n] = total.  The
// counts pass through shared memory in chunks of 8192 with coalesced loads and
// stores; each thread scans 8 consecutive entries of a chunk (one padding word per
// 32, so those reads fall on distinct banks) and a running carry links the chunks.
__global__ void __launch_bounds__(1024) k_tile_scan(const int* __restrict__ counts, int n, int* __restrict__ offs,
                                                    int* __restrict__ cursor) {
    constexpr int K = 8, CH = 1024 * K;
    __shared__ int buf[CH + CH / 32];
    __shared__ int part[1024];
    auto at = [](int i) { return i + (i >> 5); };
    int carry = 0;  // identical in every thread
    for (int base = 0; base < n; base += CH) {
        const int m = min(CH, n - base);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = threadIdx.x + k * 1024;
            buf[at(i)] = i < m ? counts[base + i] : 0;
        }
        __syncthreads();
        int v[K], sum = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            v[j] = buf[at(K * threadIdx.x + j)];
            sum += v[j];
        }
        part[threadIdx.x] = sum;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {  // inclusive Hillis-Steele scan of the partial sums
            const int u = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
            __syncthreads();
            part[threadIdx.x] += u;
            __syncthreads();
        }
        int run = carry + part[threadIdx.x] - sum;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            buf[at(K * threadIdx.x + j)] = run;
            run += v[j];
        }
        carry += part[1023];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = threadIdx.x + k * 1024;
            if (i < m) {
                const int o = buf[at(i)];
                offs[base + i] = o;
                cursor[base + i] = o;
            }
        }
        __syncthreads();  // buf and part are reused by the next chunk
    }
    if (threadIdx.x == 0) offs[n] = carry;
}

__global__ void __launch_bounds__(256) k_tile_fill(const int* __restrict__ tile_of, int64_t n,
                                                   int* __restrict__ cursor, int* __restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int t = tile_of[i];
        if (t >= 0) perm[atomicAdd(cursor + t, 1)] = (int)i;
    }
}

constexpr int kDepositBatch = 256;  // points staged per round (one per thread)
constexpr size_t deposit_smem(int p) {
    return ((size_t)(SB + p - 1) * (SB + p - 1) * (SB + p - 1) + (size_t)kDepositBatch * (3 * p + 1)) * sizeof(float);
}

// One block per tile: the tile's points deposit into a shared (SB+P-1)^3 region with
// shared-memory atomics.  Points are taken in batches of 256: each thread evaluates
// the node rule of one point into shared memory, then the P*P (a, b) columns of a
// point go to consecutive threads, each adding its P values along z.  For P = 4 the
// 16 columns of a point lie on 16 distinct banks (row stride RB = 19, plane stride
// 361 = 9 mod 32), so a warp's atomics (two points) conflict at most two ways.
template <int P>
__global__ void __launch_bounds__(256) k_tile_deposit(const float* __restrict__ pos, const float* __restrict__ w,
                                                      const int* __restrict__ perm, const int* __restrict__ offs,
                                                      float s, int N, int wrap, int NT, float* __restrict__ regions) {
    constexpr int RB = SB + P - 1, R3 = RB * RB * RB, PP = P * P, BATCH = kDepositBatch;
    // dynamic shared memory: the region, then the staged weights and offsets
    extern __shared__ float dsm[];
    float* reg = dsm;                                                   // [R3]
    float(*sw)[3 * P] = reinterpret_cast<float(*)[3 * P]>(dsm + R3);   // [BATCH][3P]: w_i bx[a], by[b], bz[c]
    int* soff = reinterpret_cast<int*>(dsm + R3 + BATCH * 3 * P);      // [BATCH]: region offset of the first node
    const int t = blockIdx.x;
    const int tx = t / (NT * NT), ty = (t / NT) % NT, tz = t % NT;
    const int msk = N - 1;
    for (int e = threadIdx.x; e < R3; e += blockDim.x) reg[e] = 0.0f;
    const int lo = offs[t], hi = offs[t + 1];
    for (int base = lo; base < hi; base += BATCH) {
        const int nb = min(BATCH, hi - base);
        if (threadIdx.x < nb) {
            const int i = perm[base + threadIdx.x];
            float bx[P], by[P], bz[P];
            int fx, fy, fz;
            node_rule<P>(__ldg(pos + 3 * i), s, N, wrap, fx, bx);
            node_rule<P>(__ldg(pos + 3 * i + 1), s, N, wrap, fy, by);
            node_rule<P>(__ldg(pos + 3 * i + 2), s, N, wrap, fz, bz);
            const float wi = w ? __ldg(w + i) : 1.0f;
            float* row = sw[threadIdx.x];
#pragma unroll
            for (int o = 0; o < P; ++o) {
                row[o] = wi * bx[o];
                row[P + o] = by[o];
                row[2 * P + o] = bz[o];
            }
            soff[threadIdx.x] = (((fx & msk) - tx * SB) * RB + ((fy & msk) - ty * SB)) * RB + ((fz & msk) - tz * SB);
        }
        __syncthreads();  // staged weights visible (and, the first time, the cleared region)
        for (int e = threadIdx.x; e < nb * PP; e += blockDim.x) {
            const int kp = e / PP, ab = e % PP, a = ab / P, b = ab % P;
            const float* wt = sw[kp];
            const float wab = wt[a] * wt[P + b];
            float* row = reg + soff[kp] + (a * RB + b) * RB;
#pragma unroll
            for (int c = 0; c < P; ++c) atomicAdd(row + c, wab * wt[2 * P + c]);
        }
        __syncthreads();  // the staging slots are reused by the next batch
    }
    __syncthreads();
    float* out = regions + (size_t)t * R3;
    for (int e = threadIdx.x; e < R3; e += blockDim.x) out[e] = reg[e];
}

// grid[x,y,z] = sum over the regions covering the cell: per axis the cell's own tile
// (local l = x % SB) and the previous tile (local l + SB, when l + SB < RB).  One block
// per (x, y) row: the (x, y) part of the up to four covering region rows is set up
// once, and each thread walks z with shifts only (same summation order as the
// per-axis enumeration (x tile, y tile, z tile)).
template <int P>
__global__ void __launch_bounds__(256) k_tile_gather(const float* __restrict__ regions, int N, int NT,
                                                     float* __restrict__ grid) {
    constexpr int RB = SB + P - 1, R3 = RB * RB * RB;
    const int y = blockIdx.x, x = blockIdx.y;
    const float* row[4];
    bool use[4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int lx = x % SB + a * SB, ly = y % SB + b * SB;
            const int tx = a ? (x / SB + NT - 1) % NT : x / SB, ty = b ? (y / SB + NT - 1) % NT : y / SB;
            use[2 * a + b] = lx < RB && ly < RB;
            row[2 * a + b] = regions + (size_t)(tx * NT + ty) * NT * R3 + (size_t)(lx * RB + ly) * RB;
        }
    float* out = grid + ((size_t)x * N + y) * N;
    for (int z = threadIdx.x; z < N; z += blockDim.x) {
        const int tz = z / SB, lz = z % SB;
        const int tzp = (tz == 0 ? NT : tz) - 1;  // previous z tile
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!use[k]) continue;  // uniform across the block
            acc += __ldg(row[k] + (size_t)tz * R3 + lz);
            if (lz + SB < RB) acc += __ldg(row[k] + (size_t)tzp * R3 + lz + SB);
        }
        out[z] = acc;
    }
}

// Node rule of every point, for inspection: first node (mod N) and the p basis
// values per axis; err bit 1 marks a rejected coordinate.
template <int P>
__global__ void __launch_bounds__(256) k_nodes(const float* __restrict__ pos, int64_t n, float s, int N, int wrap,
                                               int* __restrict__ first, float* __restrict__ wts,
                                               unsigned* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float b[P];
        int f = 0;
        const bool ok = node_rule<P>(pos[3 * i + d], s, N, wrap, f, b);
        if (!ok) atomicOr(err, 1u);
        first[3 * i + d] = ok ? (f & (N - 1)) : -1;
#pragma unroll
        for (int o = 0; o < P; ++o) wts[(3 * i + d) * P + o] = ok ? b[o] : 0.0f;
    }
}

// offs == nullptr: one catalogue of n points.  Otherwise blockIdx.y = catalogue
// c over points [offs[c], offs[c+1]), partials at part + c * 2 * gridDim.x.
__global__ void __launch_bounds__(256) k_weight_sums(const float* __restrict__ w, int64_t n,
                                                     const int64_t* __restrict__ offs, double* __restrict__ part) {
    __shared__ double red[8];
    if (offs) {
        const int64_t lo = offs[blockIdx.y];
        n = offs[blockIdx.y + 1] - lo;
        if (w) w += lo;
        part += (size_t)blockIdx.y * 2 * gridDim.x;
    }
    double s1 = 0.0, s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = w ? (double)__ldg(w + i) : 1.0;
        s1 += v;
        s2 += v * v;
    }
    double t1 = block_sum_double(s1, red);
    double t2 = block_sum_double(s2, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t1;
        part[gridDim.x + blockIdx.x] = t2;
    }
}

// p <= 4: every thread accumulates the whole table (P^3 <= 64 floats) over its own
// points as the outer product w_i^2 s_x (x) s_y (x) s_z, with no shared staging;
// the block then reduces entry by entry (warp shuffles, then the warps in a fixed
// order).  Same output layout as k_selfpair.
template <int P>
__global__ void __launch_bounds__(256) k_selfpair_reg(const float* __restrict__ pos, const float* __restrict__ w,
                                                      int64_t n, const int64_t* __restrict__ offs, float s, int N,
                                                      double* __restrict__ part) {
    constexpr int P3 = P * P * P;
    if (offs) {  // batched: blockIdx.y = catalogue, as k_weight_sums
        const int64_t lo = offs[blockIdx.y];
        n = offs[blockIdx.y + 1] - lo;
        pos += 3 * lo;
        if (w) w += lo;
        part += (size_t)blockIdx.y * P3 * gridDim.x;
    }
    __shared__ double tot[8][P3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float acc[P3];
#pragma unroll
    for (int e = 0; e < P3; ++e) acc[e] = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float b[3][P], sv[3][P];
        int f;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) ok &= node_rule<P>(__ldg(pos + 3 * i + d), s, N, 1, f, b[d]);
        const float wi = w ? __ldg(w + i) : 1.0f;
        const float w2 = ok ? wi * wi : 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int a = 0; a < P; ++a) {
                float sacc = 0.0f;
#pragma unroll
                for (int o = 0; o + a < P; ++o) sacc = fmaf(b[d][o], b[d][o + a], sacc);
                sv[d][a] = sacc;
            }
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const float xa = w2 * sv[0][a];
#pragma unroll
            for (int bb = 0; bb < P; ++bb) {
                const float xab = xa * sv[1][bb];
#pragma unroll
                for (int c = 0; c < P; ++c) acc[(a * P + bb) * P + c] = fmaf(xab, sv[2][c], acc[(a * P + bb) * P + c]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < P3; ++e) {
        float v = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) tot[wid][e] = (double)v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P3; e += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += tot[q][e];
        part[(size_t)e * gridDim.x + blockIdx.x] = t;
    }
}

// Self-pair overlap table (p > 4).  Each warp stages 32 points' per-axis overlaps in
// shared memory; every lane owns table entries e = lane + 32k and accumulates
// them over the staged points (float32), then the block sums in float64.
template <int P>
__global__ void __launch_bounds__(256) k_selfpair(const float* __restrict__ pos, const float* __restrict__ w,
                                                  int64_t n, const int64_t* __restrict__ offs, float s, int N,
                                                  double* __restrict__ part) {
    constexpr int P3 = P * P * P;
    if (offs) {  // batched: blockIdx.y = catalogue, as k_weight_sums
        const int64_t lo = offs[blockIdx.y];
        n = offs[blockIdx.y + 1] - lo;
        pos += 3 * lo;
        if (w) w += lo;
        part += (size_t)blockIdx.y * P3 * gridDim.x;
    }
    constexpr int E = (P3 + 31) / 32;
    constexpr int STRIDE = 3 * P + 1;
    __shared__ float stage[8][32][STRIDE];
    __shared__ double tot[P3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float acc[E];
#pragma unroll
    for (int k = 0; k < E; ++k) acc[k] = 0.0f;
    const int64_t nwarps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    for (int64_t base = gw * 32; base < n; base += nwarps_total * 32) {
        const int64_t i = base + lane;
        float* my = stage[wid][lane];
        if (i < n) {
            float b[3][P];
            int f;
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) ok &= node_rule<P>(__ldg(pos + 3 * i + d), s, N, 1, f, b[d]);
            const float wi = w ? __ldg(w + i) : 1.0f;
            my[0] = ok ? wi * wi : 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    float sacc = 0.0f;
#pragma unroll
                    for (int o = 0; o + a < P; ++o) sacc = fmaf(b[d][o], b[d][o + a], sacc);
                    my[1 + d * P + a] = sacc;
                }
            }
        } else {
            my[0] = 0.0f;
#pragma unroll
            for (int q = 1; q < STRIDE; ++q) my[q] = 0.0f;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int e = lane + 32 * k;
            if (e < P3) {
                const int a = e / (P * P), bb = (e / P) % P, c = e % P;
                float sacc = 0.0f;
                for (int j = 0; j < 32; ++j) {
                    const float* q = stage[wid][j];
                    sacc = fmaf(q[0] * q[1 + a], q[1 + P + bb] * q[1 + 2 * P + c], sacc);
                }
                acc[k] += sacc;
            }
        }
        __syncwarp();
    }
    for (int e = threadIdx.x; e < P3; e += blockDim.x) tot[e] = 0.0;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < nw; ++q) {  // warps add in turn: fixed order, no atomics
        if (wid == q) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int e = lane + 32 * k;
                if (e < P3) tot[e] += (double)acc[k];
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < P3; e += blockDim.x) part[(size_t)e * gridDim.x + blockIdx.x] = tot[e];
}

// Sum of one row by a block of kReduceThreads threads in a fixed order: each thread
// keeps 8 independent partial sums (8 loads in flight instead of one dependent
// chain), combined pairwise, then a block reduction.  Result valid in thread 0.
constexpr int kReduceThreads = 1024;
__device__ __forceinline__ double row_sum(const double* __restrict__ row, int cols, double* red) {
    constexpr int U = 8, B = kReduceThreads;
    double a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) a[j] = 0.0;
    int c = threadIdx.x;
    for (; c + (U - 1) * B < cols; c += U * B) {
#pragma unroll
        for (int j = 0; j < U; ++j) a[j] += row[c + j * B];
    }
    for (; c < cols; c += B) a[0] += row[c];
    const double s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    return block_sum_double(s, red);
}

// out[r] = sum_c part[r*cols + c], one block per row (deterministic order).
__global__ void __launch_bounds__(kReduceThreads) k_reduce_rows(const double* __restrict__ part, int cols,
                                                                double* __restrict__ out) {
    __shared__ double red[kReduceThreads / 32];
    const double s = row_sum(part + (size_t)blockIdx.x * cols, cols, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Row r of part (cols wide) summed into out[(r / S) * out_stride + r % S]: the
// rows of a batched launch are [catalogue][window] and land in a [catalogue][...]
// result array.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_rows_strided(const double* __restrict__ part, int cols,
                                                                        int S, double* __restrict__ out,
                                                                        int out_stride) {
    __shared__ double red[kReduceThreads / 32];
    const double s = row_sum(part + (size_t)blockIdx.x * cols, cols, red);
    if (threadIdx.x == 0) out[(size_t)(blockIdx.x / S) * out_stride + blockIdx.x % S] = s;
}

// Per catalogue c (one block each): scal[c*SCAL_STRIDE + 0..2] = sum w, sum w^2,
// N^3 / sum w; float copy of its self-pair table at stab_f + c*STAB_STRIDE.
__global__ void __launch_bounds__(256) k_finish_batch(const double* __restrict__ sums, const double* __restrict__ sp,
                                                      int p3, float* __restrict__ stab_f, int N,
                                                      double* __restrict__ scal) {
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        const double sw = sums[2 * c];
        scal[(size_t)c * SCAL_STRIDE + 0] = sw;
        scal[(size_t)c * SCAL_STRIDE + 1] = sums[2 * c + 1];
        scal[(size_t)c * SCAL_STRIDE + 2] = (double)N * (double)N * (double)N / sw;
    }
    for (int e = threadIdx.x; e < p3; e += blockDim.x) stab_f[(size_t)c * STAB_STRIDE + e] = (float)sp[(size_t)c * p3 + e];
}

// xi of every (catalogue, window): out[c*nwin + w] = dd/N^6 - sn/eps_bar_c^2,
// eps_bar_c = sum w_c / N^3 (dd, sn laid out like out; sn is already / N^6).
__global__ void __launch_bounds__(256) k_xi_batch_finish(const double* __restrict__ dd, const double* __restrict__ sn,
                                                         const double* __restrict__ scal, int ncat, int nwin, int N,
                                                         double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncat * nwin) return;
    const int c = i / nwin;
    const double n3 = (double)N * N * N, n6 = n3 * n3;
    const double eb = scal[(size_t)c * SCAL_STRIDE] / n3;
    out[i] = dd[i] / n6 - sn[i] / (eb * eb);
}

// scal[0] = sum w, scal[1] = sum w^2, scal[2] = N^3 / sum w (the inverse mean);
// float copy of the self-pair table for the window kernels.
__global__ void k_finish_field(const double* __restrict__ sums, const double* __restrict__ stab_d, int p3,
                               float* __restrict__ stab_f, int N, double* __restrict__ scal) {
    if (threadIdx.x == 0) {
        scal[0] = sums[0];
        scal[1] = sums[1];
        scal[2] = (double)N * (double)N * (double)N / sums[0];
    }
    for (int e = threadIdx.x; e < p3; e += blockDim.x) stab_f[e] = (float)stab_d[e];
}

static int nblocks_for(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_scatter(int N, int p, const float* pos, const float* w, int64_t n, float* grid, float s,
                           int wrap, unsigned* err, cudaStream_t st, const Tracer& tr) {
    if (n == 0) return cudaSuccess;
    const int nb = nblocks_for(n, 256, 148 * 32);
    tr(K_SCATTER, 0, st);
    switch (p) {
#define HERMES_SC(P) \
    case P: k_scatter<P><<<nb, 256, 0, st>>>(pos, w, n, grid, s, N, wrap, err); break;
        HERMES_SC(1) HERMES_SC(2) HERMES_SC(3) HERMES_SC(4) HERMES_SC(5) HERMES_SC(6) HERMES_SC(7) HERMES_SC(8)
#undef HERMES_SC
        default: return cudaErrorInvalidValue;
    }
    tr(K_SCATTER, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_nodes(int N, int p, const float* pos, int64_t n, float s, int wrap, int* first, float* wts,
                         unsigned* err, cudaStream_t st, const Tracer& tr) {
    if (n == 0) return cudaSuccess;
    const int nb = (int)((n + 255) / 256);
    tr(K_NODES, 0, st);
    switch (p) {
#define HERMES_ND(P) \
    case P: k_nodes<P><<<nb, 256, 0, st>>>(pos, n, s, N, wrap, first, wts, err); break;
        HERMES_ND(1) HERMES_ND(2) HERMES_ND(3) HERMES_ND(4) HERMES_ND(5) HERMES_ND(6) HERMES_ND(7) HERMES_ND(8)
#undef HERMES_ND
        default: return cudaErrorInvalidValue;
    }
    tr(K_NODES, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_scatter_batch(int N, int p, const float* pos, const float* w, const int64_t* offs, int c0, int c1,
                                 int64_t n_max, float* grid, float s, int wrap, unsigned* err, cudaStream_t st,
                                 const Tracer& tr) {
    if (c0 < 0 || c1 <= c0 || c1 - c0 > MAX_CATALOGUES) return cudaErrorInvalidValue;
    const int nb = nblocks_for(n_max, 256, 148 * 32);
    tr(K_SCATTER, 0, st);
    switch (p) {
#define HERMES_SC(P) \
    case P: k_scatter_batch<P><<<nb, 256, 0, st>>>(pos, w, offs, c0, c1, grid, s, N, wrap, err); break;
        HERMES_SC(1) HERMES_SC(2) HERMES_SC(3) HERMES_SC(4) HERMES_SC(5) HERMES_SC(6) HERMES_SC(7) HERMES_SC(8)
#undef HERMES_SC
        default: return cudaErrorInvalidValue;
    }
    tr(K_SCATTER, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_weight_sums(const float* w, int64_t n, double* part, int nblk, cudaStream_t st, const Tracer& tr,
                               const int64_t* offs, int ncat) {
    tr(K_WEIGHT_SUMS, 0, st);
    k_weight_sums<<<dim3(nblk, offs ? ncat : 1), 256, 0, st>>>(w, n, offs, part);
    tr(K_WEIGHT_SUMS, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_selfpair(int N, int p, const float* pos, const float* w, int64_t n, float s, double* part,
                            int nblk, cudaStream_t st, const Tracer& tr, const int64_t* offs, int ncat) {
    tr(K_SELFPAIR, 0, st);
    const dim3 g(nblk, offs ? ncat : 1);
    switch (p) {
#define HERMES_SPR(P) \
    case P: k_selfpair_reg<P><<<g, 256, 0, st>>>(pos, w, n, offs, s, N, part); break;
#define HERMES_SP(P) \
    case P: k_selfpair<P><<<g, 256, 0, st>>>(pos, w, n, offs, s, N, part); break;
        HERMES_SPR(1) HERMES_SPR(2) HERMES_SPR(3) HERMES_SPR(4) HERMES_SP(5) HERMES_SP(6) HERMES_SP(7) HERMES_SP(8)
#undef HERMES_SPR
#undef HERMES_SP
        default: return cudaErrorInvalidValue;
    }
    tr(K_SELFPAIR, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_reduce_rows(const double* part, int rows, int cols, double* out, cudaStream_t st,
                               const Tracer& tr) {
    if (rows <= 0) return cudaSuccess;
    tr(K_REDUCE, 0, st);
    k_reduce_rows<<<rows, kReduceThreads, 0, st>>>(part, cols, out);
    tr(K_REDUCE, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_finish_field(const double* sums, const double* stab_d, int p3, float* stab_f, int N,
                                double* scal, cudaStream_t st, const Tracer& tr) {
    tr(K_FINISH, 0, st);
    k_finish_field<<<1, 256, 0, st>>>(sums, stab_d, p3, stab_f, N, scal);
    tr(K_FINISH, 1, st);
    return cudaGetLastError();
}

// Delta = (eps_D - alpha eps_R) / eps_bar_D in place, 4 cells per thread (n is a
// multiple of 4: N^3 with N >= 16); block 0 also writes the combined self-pair table.
__global__ void __launch_bounds__(256) k_combine_randoms(float4* __restrict__ grid, const float4* __restrict__ rgrid,
                                                         size_t n4, float alpha, float inv_ebar,
                                                         const double* __restrict__ stab_d,
                                                         const double* __restrict__ rstab_d, double alpha2,
                                                         float* __restrict__ stab_f, int p3) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 d = grid[i], r = __ldg(rgrid + i);
        grid[i] = make_float4(fmaf(-alpha, r.x, d.x) * inv_ebar, fmaf(-alpha, r.y, d.y) * inv_ebar,
                              fmaf(-alpha, r.z, d.z) * inv_ebar, fmaf(-alpha, r.w, d.w) * inv_ebar);
    }
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < p3; e += blockDim.x) stab_f[e] = (float)(stab_d[e] + alpha2 * rstab_d[e]);
}

cudaError_t launch_combine_randoms(float* grid, const float* rgrid, size_t n, float alpha, float inv_ebar,
                                   const double* stab_d, const double* rstab_d, double alpha2, float* stab_f, int p3,
                                   cudaStream_t st, const Tracer& tr) {
    tr(K_COMBINE, 0, st);
    k_combine_randoms<<<148 * 8, 256, 0, st>>>(reinterpret_cast<float4*>(grid), reinterpret_cast<const float4*>(rgrid),
                                               n / 4, alpha, inv_ebar, stab_d, rstab_d, alpha2, stab_f, p3);
    tr(K_COMBINE, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_reduce_rows_strided(const double* part, int rows, int cols, int S, double* out, int out_stride,
                                       cudaStream_t st, const Tracer& tr) {
    if (rows <= 0) return cudaSuccess;
    tr(K_REDUCE, 0, st);
    k_reduce_rows_strided<<<rows, kReduceThreads, 0, st>>>(part, cols, S, out, out_stride);
    tr(K_REDUCE, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_finish_batch(const double* sums, const double* sp, int p3, float* stab_f, int N, double* scal,
                                int ncat, cudaStream_t st, const Tracer& tr) {
    tr(K_FINISH, 0, st);
    k_finish_batch<<<ncat, 256, 0, st>>>(sums, sp, p3, stab_f, N, scal);
    tr(K_FINISH, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_xi_batch_finish(const double* dd, const double* sn, const double* scal, int ncat, int nwin, int N,
                                   double* out, cudaStream_t st, const Tracer& tr) {
    const int n = ncat * nwin;
    tr(K_FINISH, 0, st);
    k_xi_batch_finish<<<(n + 255) / 256, 256, 0, st>>>(dd, sn, scal, ncat, nwin, N, out);
    tr(K_FINISH, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_gather_marks(int N, int p, const float* pos, int64_t n, const float* field, float s, int wrap,
                                int kind, float a, float b, float self, float* out, unsigned* err, cudaStream_t st,
                                const Tracer& tr) {
    if (n == 0) return cudaSuccess;
    const int nb = nblocks_for(n, 256, 148 * 16);
    tr(K_GATHER, 0, st);
    switch (p) {
#define HERMES_GM(P) \
    case P: k_gather_marks<P><<<nb, 256, 0, st>>>(pos, n, field, s, N, wrap, kind, a, b, self, out, err); break;
        HERMES_GM(1) HERMES_GM(2) HERMES_GM(3) HERMES_GM(4) HERMES_GM(5) HERMES_GM(6) HERMES_GM(7) HERMES_GM(8)
#undef HERMES_GM
        default: return cudaErrorInvalidValue;
    }
    tr(K_GATHER, 1, st);
    return cudaGetLastError();
}

size_t scatter_tiled_region_floats(int N, int p) {
    const int NT = N / SB, RB = SB + p - 1;
    return (size_t)NT * NT * NT * RB * RB * RB;
}
int scatter_tiled_tiles(int N) { return (N / SB) * (N / SB) * (N / SB); }

cudaError_t launch_scatter_tiled(int N, int p, const float* pos, const float* w, int64_t n, float* grid, float s,
                                 int wrap, unsigned* err, int* tile_of, int* perm, int* counts, int* offs,
                                 int* cursor, float* regions, cudaStream_t st, const Tracer& tr) {
    if (N < SB || p < 1 || p > 8 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int NT = N / SB, ntiles = NT * NT * NT;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)ntiles * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int nb = nblocks_for(n, 256, 148 * 16);
    tr(K_SCATTER, 0, st);
    switch (p) {
#define HERMES_TC(P) \
    case P: k_tile_count<P><<<nb, 256, 0, st>>>(pos, w, n, s, N, wrap, NT, counts, tile_of, err); break;
        HERMES_TC(1) HERMES_TC(2) HERMES_TC(3) HERMES_TC(4) HERMES_TC(5) HERMES_TC(6) HERMES_TC(7) HERMES_TC(8)
#undef HERMES_TC
    }
    k_tile_scan<<<1, 1024, 0, st>>>(counts, ntiles, offs, cursor);
    k_tile_fill<<<nb, 256, 0, st>>>(tile_of, n, cursor, perm);
    const dim3 ng((unsigned)N, (unsigned)N);  // one block per (x, y) row
    const int gt = N < 256 ? N : 256;
    switch (p) {
#define HERMES_TD(P)                                                                                    \
    case P:                                                                                             \
        if (deposit_smem(P) > 48 * 1024 &&                                                              \
            (e = cudaFuncSetAttribute(k_tile_deposit<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                      (int)deposit_smem(P))) != cudaSuccess)                             \
            return e;                                                                                   \
        k_tile_deposit<P><<<ntiles, 256, deposit_smem(P), st>>>(pos, w, perm, offs, s, N, wrap, NT, regions); \
        k_tile_gather<P><<<ng, gt, 0, st>>>(regions, N, NT, grid);                                      \
        break;
        HERMES_TD(1) HERMES_TD(2) HERMES_TD(3) HERMES_TD(4) HERMES_TD(5) HERMES_TD(6) HERMES_TD(7) HERMES_TD(8)
#undef HERMES_TD
    }
    tr(K_SCATTER, 1, st);
    return cudaGetLastError();
}

}  // namespace hermes
