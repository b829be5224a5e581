// Interface metrics (arXiv 2504.10539 Sec. II-D Eqs. 9-13, discretised in
// Sec. IV-E Eqs. 14-16), the mass, the Laplace measurement, and the interface
// correction (Sec. II-C step 3), for every lattice of a job table.
//
// Segmented, deterministic two-level reductions: lattice j owns red_blocks(j)
// virtual blocks (a function of its size only); virtual block b of lattice j
// accumulates FP64 partial sums / extrema over cells b*256+t, b*256+t+R*256, ...
// (R = red_blocks(j)), reduces them by a fixed warp-shuffle tree into one partial,
// and one block per lattice folds that lattice's partials in block order.  The
// result depends on the lattice alone: it is the same whatever else is in the
// table and however the persistent grid is scheduled, so repeated runs are
// bit-identical and a lattice gives the same numbers alone and in a batch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

constexpr int RED_GRID = 152 * 8;  // persistent grid of the reduction kernels

// Reduction blocks of a lattice: about RB_CELLS_PER_THREAD cells per thread, so that the
// per-block tree (and its FP64 folds) is amortised over many cells.
int red_blocks_for(long long cells) {
    long long b = (cells + RB_THREADS * RB_CELLS_PER_THREAD - 1) / (RB_THREADS * RB_CELLS_PER_THREAD);
    if (b > RB_MAX_BLOCKS) b = RB_MAX_BLOCKS;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ int find_blk(const int* __restrict__ pre, int n, int v) {
    int lo = 0, hi = n;  // pre[lo] <= v < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Block reduction of FP32 partials (FP32 and FP16-offset lattices).  The FP64 pipe of this part
// runs at a small fraction of the FP32 rate, so the per-block tree stays in FP32: a sum as an
// unevaluated pair hi + lo merged by an error-free TwoSum (about 2^-48 relative), an extremum or
// a count (an integer below 2^24, so exact) directly; thread 0 converts the results to FP64.
// Fixed tree, as in block_reduce: the result depends on the block's values alone.
__device__ __forceinline__ void ff_merge(float& hi, float& lo, float bhi, float blo) {
    const float s = __fadd_rn(hi, bhi);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bhi, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, blo), e);
}
template <int NV>
__device__ __forceinline__ void ff_level(float (&hi)[NV], float (&lo)[NV], const int (&op)[NV], int o) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float bh = __shfl_down_sync(0xffffffffu, hi[k], o);
        const float bl = __shfl_down_sync(0xffffffffu, lo[k], o);
        if (op[k] == 0) ff_merge(hi[k], lo[k], bh, bl);
        else hi[k] = op[k] == 1 ? fmaxf(hi[k], bh) : fminf(hi[k], bh);
    }
}
// op: 0 = sum, 1 = max, 2 = min (lo unused).  out valid in thread 0; smem: 2 NV x 32 floats.
template <int NV>
__device__ __forceinline__ void block_reduce_ff(float (&hi)[NV], float (&lo)[NV], const int (&op)[NV], float* smem,
                                                double (&out)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ff_level<NV>(hi, lo, op, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int k = 0; k < NV; ++k) {
            smem[k * 32 + warp] = hi[k];
            smem[(NV + k) * 32 + warp] = lo[k];
        }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float init = op[k] == 0 ? 0.0f : (op[k] == 1 ? -INFINITY : INFINITY);
            hi[k] = lane < nw ? smem[k * 32 + lane] : init;
            lo[k] = lane < nw ? smem[(NV + k) * 32 + lane] : 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ff_level<NV>(hi, lo, op, o);
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = op[k] == 0 ? (double)hi[k] + (double)lo[k] : (double)hi[k];
    }
    __syncthreads();
}

// Virtual block vb of the table -> lattice j, local block lb.
struct BlkMap {
    int j, lb;
};
__device__ __forceinline__ BlkMap map_blk(const TableView& t, int n, int vb) {
    BlkMap m;
    m.j = find_blk(t.blk_pre, n, vb);
    m.lb = vb - t.blk_pre[m.j];
    return m;
}

// Cell index c = y nx + x of a grid-stride loop together with its coordinates, advanced by a
// fixed stride (stride = sy nx + sx, 0 <= sx < nx) without a division per cell.
struct CellIt {
    long long c, stride;
    int x, y, sx, sy;
    __device__ __forceinline__ CellIt(long long c0, long long stride_, int nx) : c(c0), stride(stride_) {
        x = (int)(c0 % nx);
        y = (int)(c0 / nx);
        sx = (int)(stride_ % nx);
        sy = (int)(stride_ / nx);
    }
    __device__ __forceinline__ void next(int nx) {
        c += stride;
        x += sx;
        y += sy;
        if (x >= nx) {
            x -= nx;
            ++y;
        }
    }
    __device__ __forceinline__ long long pop_offset(int pitch) const { return (long long)y * pitch + x; }
};

// ---------------------------------------------------------------------------------------------
// Per-array kernels (one lattice given by raw pointers), used by pl_metrics_noalloc.

// Threshold for "g > thr" in the arithmetic type R: for FP32 g, g > thr (FP64) holds exactly
// when g > the largest FP32 number <= thr, so the count is the one an FP64 comparison gives.
template <typename R>
__device__ __forceinline__ R threshold_below(double thr);
template <>
__device__ __forceinline__ double threshold_below<double>(double thr) { return thr; }
template <>
__device__ __forceinline__ float threshold_below<float>(double thr) { return __double2float_rd(thr); }

// Per-thread metric accumulator: {sum rho, max g, sum g, sum g^2, max rho, min rho,
// count(g > thr), count(non-physical rho)}; sums in SumAcc, extrema and counts exact.
template <typename R>
struct GradAcc {
    SumAcc<R> mass, sum_g, sum_g2;
    R gmax = R(0), rmax = R(-INFINITY), rmin = R(INFINITY);
    unsigned count = 0, bad = 0;
    __device__ __forceinline__ void to(double (&v)[8]) const {
        v[0] = mass.value();
        v[1] = (double)gmax;
        v[2] = sum_g.value();
        v[3] = sum_g2.value();
        v[4] = (double)rmax;
        v[5] = (double)rmin;
        v[6] = (double)count;
        v[7] = (double)bad;
    }
};

// Eq. 16 gradient magnitude (central differences, periodic, dx = dy = 1) of cell c = (x, y),
// optionally stored to g, accumulated into a (a non-physical cell: rho <= 0 or not finite).
// The five densities the Eq. 16 gradient magnitude of cell c = (x, y) reads (periodic).
template <typename R>
struct GradIn {
    R xp, xm, yp, ym, r;
};
template <typename R>
__device__ __forceinline__ GradIn<R> grad_load(const R* __restrict__ rho, int nx, int ny, long long c, int x, int y) {
    const long long row = c - x;
    return GradIn<R>{rho[row + (x == nx - 1 ? 0 : x + 1)], rho[row + (x == 0 ? nx - 1 : x - 1)],
                     rho[(long long)(y == ny - 1 ? 0 : y + 1) * nx + x], rho[(long long)(y == 0 ? ny - 1 : y - 1) * nx + x],
                     rho[c]};
}
// Eq. 16 gradient magnitude (central differences, dx = dy = 1) of cell c from its loaded
// densities, optionally stored to g, accumulated into a (a non-physical cell: rho <= 0 or not
// finite).
template <typename R>
__device__ __forceinline__ void grad_apply(const GradIn<R>& in, long long c, R* __restrict__ g, R thr, GradAcc<R>& a) {
    const R gx = (in.xp - in.xm) / R(2);
    const R gy = (in.yp - in.ym) / R(2);
    const R gm = sqrt(gx * gx + gy * gy);
    if (g) g[c] = gm;
    const R r = in.r;
    a.mass.add(r);
    a.gmax = fmax(a.gmax, gm);
    a.sum_g.add(gm);
    a.sum_g2.add_prod(gm, gm);
    a.rmax = fmax(a.rmax, r);
    a.rmin = fmin(a.rmin, r);
    a.count += gm > thr ? 1u : 0u;
    a.bad += (r > R(0) && isfinite(r)) ? 0u : 1u;
}
template <typename R>
__device__ __forceinline__ void grad_accumulate(const R* __restrict__ rho, int nx, int ny, long long c, int x, int y,
                                                R* __restrict__ g, R thr, GradAcc<R>& a) {
    grad_apply(grad_load(rho, nx, ny, c, x, y), c, g, thr, a);
}

// A thread's cells, U at a time: the next U cells of the walk (valid while c < N) with their
// loads issued together, then processed in walk order, so that the sums are the same as cell
// by cell while U times the loads per thread are in flight (U = 2 measured best of 1, 2, 4, 8:
// more cells per thread cost resident warps through registers).
constexpr int CELL_BATCH = 2;
struct CellBatch {
    long long c[CELL_BATCH];
    int x[CELL_BATCH], y[CELL_BATCH];
    bool v[CELL_BATCH];
    __device__ __forceinline__ void take(CellIt& it, long long N, int nx) {
#pragma unroll
        for (int u = 0; u < CELL_BATCH; ++u) {
            v[u] = it.c < N;
            c[u] = it.c;
            x[u] = it.x;
            y[u] = it.y;
            if (v[u]) it.next(nx);
        }
    }
};

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_grad_reduce(const R* __restrict__ rho, int nx, int ny,
                                                            R* __restrict__ g, double threshold,
                                                            double* __restrict__ partials) {
    __shared__ double sm[8 * 32];
    const long long N = (long long)nx * ny;
    GradAcc<R> a;
    const R thr = threshold_below<R>(threshold);
    for (CellIt it(blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, nx); it.c < N;
         it.next(nx))
        grad_accumulate(rho, nx, ny, it.c, it.x, it.y, g, thr, a);
    double v[8];
    const int op[8] = {0, 1, 0, 0, 1, 2, 0, 0};
    a.to(v);
    block_reduce<8>(v, op, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) partials[blockIdx.x * PARTIAL_STRIDE + k] = v[k];
}

__device__ __forceinline__ void fold_metric_partials(const double* __restrict__ partials, int nb, DevRecord* rec,
                                                     int set_mass0, double* sm) {
    double v[7] = {0.0, 0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    const int op[7] = {0, 1, 0, 0, 1, 2, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double* p = partials + b * PARTIAL_STRIDE;
        v[0] += p[0];
        v[1] = fmax(v[1], p[1]);
        v[2] += p[2];
        v[3] += p[3];
        v[4] = fmax(v[4], p[4]);
        v[5] = fmin(v[5], p[5]);
        v[6] += p[6];
    }
    block_reduce<7>(v, op, sm);
    if (threadIdx.x == 0) {
        rec->mass = v[0];
        rec->gmax = v[1];
        rec->sum_g = v[2];
        rec->sum_g2 = v[3];
        rec->rho_max = v[4];
        rec->rho_min = v[5];
        rec->count = (long long)v[6];
        rec->rho_in = v[4];   // starting estimates of the Laplace iteration
        rec->rho_out = v[5];
        // 1: record M0; 2: record M0 only where none is recorded yet (newly admitted lattices)
        if (set_mass0 == 1 || (set_mass0 == 2 && rec->mass0 == 0.0)) rec->mass0 = v[0];
    }
}

__global__ void __launch_bounds__(RB_THREADS) k_final_metrics(const double* __restrict__ partials, int nb,
                                                              DevRecord* rec, int set_mass0) {
    __shared__ double sm[7 * 32];
    fold_metric_partials(partials, nb, rec, set_mass0, sm);
}

// ---------------------------------------------------------------------------------------------
// Table kernels: metrics.

// rho = sum_i f_i and j = sum_i f_i c_i per cell, from the decoded stored state.
// Density and momentum of one cell into the moment fields, from its populations P (FP32 / FP64)
// or from its FP16 offsets h and reference terms t.  The moments pass and the correction's
// apply pass (for the cells it changed, from the values it stores) both write through these, so
// the fields hold the same values either way.
template <typename R>
__device__ __forceinline__ void put_moments(const LatDesc& d, long long c, R rho_c, const R (&P)[9]) {
    static_cast<R*>(d.rho)[c] = rho_c;
    static_cast<R*>(d.jx)[c] = (P[1] - P[3]) + (P[5] - P[6]) + (P[8] - P[7]);
    static_cast<R*>(d.jy)[c] = (P[2] - P[4]) + (P[5] + P[6]) - (P[7] + P[8]);
}
__device__ __forceinline__ void put_moments_f16(const LatDesc& d, long long c, const float (&h)[9], const float (&tt)[9]) {
    // f_i = h_i + t_i; the mass as the sum of the two exact-where-possible parts
    float P[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) P[i] = h[i] + tt[i];
    put_moments<float>(d, c, sum9(tt) + sum9(h), P);
}
template <typename R>
__device__ __forceinline__ void put_moments_p(const LatDesc& d, long long c, const R (&P)[9]) {
    put_moments<R>(d, c, ((P[0] + P[1]) + (P[2] + P[3])) + ((P[4] + P[5]) + (P[6] + P[7])) + P[8], P);
}

// The same from the stored populations.
template <int MODE>
__device__ __forceinline__ void cell_moments(const typename Traits<MODE>::S* f, const LatDesc& d, const CellIt& it) {
    using R = typename Traits<MODE>::R;
    if constexpr (MODE == PL_F16_OFFSET) {
        float h[9], tt[9];
        f16_cell(f, d.plane, d.pitch, d.nx, d.ny, it.x, it.y, h, tt);
        put_moments_f16(d, it.c, h, tt);
    } else {
        const long long o = it.pop_offset(d.pitch);
        R P[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = decode<MODE>(f[i * d.plane + o]);
        put_moments_p<R>(d, it.c, P);
    }
}

template <int MODE>
__global__ void __launch_bounds__(RB_THREADS) k_moments(TableView t, int parity) {
    using S = typename Traits<MODE>::S;
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        const S* f = static_cast<const S*>(d.pops[d.phase ^ parity]);
        const long long N = (long long)d.nx * d.ny;
        for (CellIt it((long long)m.lb * RB_THREADS + threadIdx.x, (long long)d.red_blocks * RB_THREADS, d.nx); it.c < N;
             it.next(d.nx))
            cell_moments<MODE>(f, d, it);
    }
}

// Also counts non-physical cells (rho <= 0 or not finite) in partial slot 7.
template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_grad_tab(TableView t) {
    __shared__ double sm[8 * 32];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        const long long N = (long long)d.nx * d.ny;
        const R* rho = static_cast<const R*>(d.rho);
        const R thr = threshold_below<R>(d.threshold);
        GradAcc<R> a;
        R* gout = static_cast<R*>(d.g);
        for (CellIt it((long long)m.lb * RB_THREADS + threadIdx.x, (long long)d.red_blocks * RB_THREADS, d.nx); it.c < N;) {
            CellBatch b;
            b.take(it, N, d.nx);
            GradIn<R> in[CELL_BATCH];
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u)
                if (b.v[u]) in[u] = grad_load(rho, d.nx, d.ny, b.c[u], b.x[u], b.y[u]);
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u)
                if (b.v[u]) grad_apply(in[u], b.c[u], gout, thr, a);
        }
        double v[8];
        const int op[8] = {0, 1, 0, 0, 1, 2, 0, 0};
        if constexpr (std::is_same<R, float>::value) {
            float hi[8] = {a.mass.hi, a.gmax, a.sum_g.hi, a.sum_g2.hi, a.rmax, a.rmin, (float)a.count, (float)a.bad};
            float lo[8] = {a.mass.lo, 0.0f, a.sum_g.lo, a.sum_g2.lo, 0.0f, 0.0f, 0.0f, 0.0f};
            block_reduce_ff<8>(hi, lo, op, reinterpret_cast<float*>(sm), v);
        } else {
            a.to(v);
            block_reduce<8>(v, op, sm);
        }
        if (threadIdx.x == 0)
            for (int k = 0; k < 8; ++k) d.partials[m.lb * PARTIAL_STRIDE + k] = v[k];
    }
}

// Folds the metric partials; a lattice with any non-physical cell gets the sticky status
// PL_ERR_NONPHYSICAL (its neighbours in the table are not affected).
__global__ void __launch_bounds__(RB_THREADS) k_final_metrics_tab(TableView t, int set_mass0) {
    __shared__ double sm[8 * 32];
    const int n = t.hdr->n;
    const int op1[1] = {0};
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const LatDesc& d = t.d[j];
        fold_metric_partials(d.partials, d.red_blocks, d.rec, set_mass0, sm);
        double bad[1] = {0.0};
        for (int b = threadIdx.x; b < d.red_blocks; b += blockDim.x) bad[0] += d.partials[b * PARTIAL_STRIDE + 7];
        block_reduce<1>(bad, op1, sm + 7 * 32);
        if (threadIdx.x == 0 && bad[0] > 0.0 && d.rec->status == PL_OK) d.rec->status = PL_ERR_NONPHYSICAL;
    }
}

// Laplace measurement about the droplet centre (single-droplet lattices; build-defined
// estimator, Sec. III-A set-up): R_eq = sqrt((M - N rho_out) / (pi (rho_in - rho_out)));
// inner cells d < R_eq/2, outer cells d > R_eq + 4 width; means of rho and of the bulk
// pressure p = rho/3 + G psi^2/6.
__device__ __forceinline__ double min_image_d(double d, double n) {
    double a = fabs(fmod(d, n));
    return a > 0.5 * n ? n - a : a;
}

__device__ __forceinline__ double laplace_req(const DevRecord* rec, long long N) {
    return sqrt((rec->mass - (double)N * rec->rho_out) / (3.14159265358979323846 * (rec->rho_in - rec->rho_out)));
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_laplace_region(TableView t) {
    __shared__ double sm[6 * 32];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    const int op[6] = {0, 0, 0, 0, 0, 0};
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        if (!d.has_centre) continue;
        const long long N = (long long)d.nx * d.ny;
        const double Req = laplace_req(d.rec, N);
        const R* rho = static_cast<const R*>(d.rho);
        SumAcc<R> in_rho, in_p, out_rho, out_p;  // inner / outer sums of rho and p
        unsigned in_n = 0, out_n = 0;
        // geometry and pressure in the lattice's arithmetic type, sums in SumAcc
        const R nxr = R(d.nx), nyr = R(d.ny), cxr = R(d.cx), cyr = R(d.cy), rho0 = R(d.rho0), G = R(d.G);
        const R inv_rho0 = R(1.0 / d.rho0), third = R(1.0 / 3.0), sixth = R(1.0 / 6.0);  // no divisions per cell
        const R inner = R(0.5 * Req), outer = R(Req + 4.0 * d.width);
        for (CellIt it((long long)m.lb * RB_THREADS + threadIdx.x, (long long)d.red_blocks * RB_THREADS, d.nx); it.c < N;) {
            CellBatch b;
            b.take(it, N, d.nx);
            R rr[CELL_BATCH];
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u) rr[u] = b.v[u] ? rho[b.c[u]] : R(0);
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u) {
                if (!b.v[u]) continue;
                R ax = fabs(R(b.x[u]) - cxr), ay = fabs(R(b.y[u]) - cyr);
                if (ax >= nxr) ax = fmod(ax, nxr);
                if (ay >= nyr) ay = fmod(ay, nyr);
                if (ax > R(0.5) * nxr) ax = nxr - ax;  // minimum image
                if (ay > R(0.5) * nyr) ay = nyr - ay;
                const R dd = sqrt(ax * ax + ay * ay);
                const R r = rr[u];
                const R ps = -rho0 * expm1(-r * inv_rho0);
                const R p = r * third + G * ps * ps * sixth;
                if (dd < inner) {
                    in_rho.add(r);
                    in_p.add(p);
                    ++in_n;
                }
                if (dd > outer) {
                    out_rho.add(r);
                    out_p.add(p);
                    ++out_n;
                }
            }
        }
        double v[6];
        if constexpr (std::is_same<R, float>::value) {
            float hi[6] = {in_rho.hi, in_p.hi, (float)in_n, out_rho.hi, out_p.hi, (float)out_n};
            float lo[6] = {in_rho.lo, in_p.lo, 0.0f, out_rho.lo, out_p.lo, 0.0f};
            block_reduce_ff<6>(hi, lo, op, reinterpret_cast<float*>(sm), v);
        } else {
            v[0] = in_rho.value(), v[1] = in_p.value(), v[2] = (double)in_n;
            v[3] = out_rho.value(), v[4] = out_p.value(), v[5] = (double)out_n;
            block_reduce<6>(v, op, sm);
        }
        if (threadIdx.x == 0)
            for (int k = 0; k < 6; ++k) d.partials[m.lb * PARTIAL_STRIDE + k] = v[k];
    }
}

__global__ void __launch_bounds__(RB_THREADS) k_laplace_final(TableView t) {
    __shared__ double sm[6 * 32];
    const int n = t.hdr->n;
    const int op[6] = {0, 0, 0, 0, 0, 0};
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const LatDesc& d = t.d[j];
        if (!d.has_centre) continue;
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int b = threadIdx.x; b < d.red_blocks; b += blockDim.x)
            for (int k = 0; k < 6; ++k) v[k] += d.partials[b * PARTIAL_STRIDE + k];
        block_reduce<6>(v, op, sm);
        if (threadIdx.x == 0) {
            DevRecord* rec = d.rec;
            rec->R_eq = laplace_req(rec, (long long)d.nx * d.ny);
            rec->rho_in = v[2] > 0 ? v[0] / v[2] : NAN;
            rec->p_in = v[2] > 0 ? v[1] / v[2] : NAN;
            rec->rho_out = v[5] > 0 ? v[3] / v[5] : NAN;
            rec->p_out = v[5] > 0 ? v[4] / v[5] : NAN;
        }
    }
}

template <int MODE>
static cudaError_t metrics_t(const TableView& t, int parity, int set_mass0, int laplace, int moments_current,
                             cudaStream_t s) {
    using R = typename Traits<MODE>::R;
    int launches = 2;
    if (!moments_current) {
        k_moments<MODE><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);
        ++launches;
    }
    k_grad_tab<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_final_metrics_tab<<<RED_GRID, RB_THREADS, 0, s>>>(t, set_mass0);
    if (laplace) {
        for (int it = 0; it < 2; ++it) {
            k_laplace_region<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
            k_laplace_final<<<RED_GRID, RB_THREADS, 0, s>>>(t);
        }
        launches += 4;
    }
    note_launches(launches);
    return cudaGetLastError();
}

cudaError_t launch_metrics_tab(const TableView& t, int storage, int parity, int set_mass0, int laplace,
                               cudaStream_t s, int moments_current) {
    switch (storage) {
        case PL_F64: return metrics_t<PL_F64>(t, parity, set_mass0, laplace, moments_current, s);
        case PL_F32: return metrics_t<PL_F32>(t, parity, set_mass0, laplace, moments_current, s);
        case PL_F16_OFFSET: return metrics_t<PL_F16_OFFSET>(t, parity, set_mass0, laplace, moments_current, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Interface correction (Sec. II-C step 3; the operator is the build's reading, the paper
// gives none):
//   m = g / G_max; drho_raw = beta_rho m (rho^ - rho)
//   drho = drho_raw - m (sum drho_raw + (M - M0)) / sum m;  rho' = rho + drho
//   dj_raw = beta_u m (rho' u^ - j); dj = dj_raw - m sum dj_raw / sum m;  u' = (j + dj) / rho'
//   f_i += f_i^eq(rho', u') - f_i^eq(rho, u) on cells with m > 0.

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_corr_sums1(TableView t) {
    __shared__ double sm[3 * 32];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    const int op[3] = {0, 0, 0};
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        const long long N = (long long)d.nx * d.ny;
        const R* rho = static_cast<const R*>(d.rho);
        const R* g = static_cast<const R*>(d.g);
        const R* out3 = static_cast<const R*>(d.out3);
        const R gmax = R(d.rec->gmax), beta_rho = R(d.beta_rho), eps = R(d.mask_eps);
        SumAcc<R> sm_m, sm_dr, sm_rho;  // sum m, sum drho_raw, sum rho
        const long long step = (long long)d.red_blocks * RB_THREADS;
        for (long long c0 = (long long)m.lb * RB_THREADS + threadIdx.x; c0 < N; c0 += CELL_BATCH * step) {
            R rr[CELL_BATCH], gg[CELL_BATCH], oo[CELL_BATCH];   // loads of U cells together
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u) {
                const long long c = c0 + u * step;
                const bool v = c < N;
                rr[u] = v ? rho[c] : R(0);
                gg[u] = v ? g[c] : R(0);
                oo[u] = v ? out3[c] : R(0);
            }
#pragma unroll
            for (int u = 0; u < CELL_BATCH; ++u) {
                if (c0 + u * step >= N) break;
                const R r = rr[u];
                R mm = gmax > R(0) ? gg[u] / gmax : R(0);
                if (!(mm > eps)) mm = R(0);   // outside the interface band (the network is not read there)
                sm_m.add(mm);
                sm_dr.add(mm > R(0) ? beta_rho * mm * (oo[u] - r) : R(0));
                sm_rho.add(r);
            }
        }
        double v[3];
        if constexpr (std::is_same<R, float>::value) {
            float hi[3] = {sm_m.hi, sm_dr.hi, sm_rho.hi}, lo[3] = {sm_m.lo, sm_dr.lo, sm_rho.lo};
            block_reduce_ff<3>(hi, lo, op, reinterpret_cast<float*>(sm), v);
        } else {
            v[0] = sm_m.value(), v[1] = sm_dr.value(), v[2] = sm_rho.value();
            block_reduce<3>(v, op, sm);
        }
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) d.partials[m.lb * PARTIAL_STRIDE + k] = v[k];
    }
}

__global__ void __launch_bounds__(RB_THREADS) k_corr_final1(TableView t) {
    __shared__ double sm[3 * 32];
    const int n = t.hdr->n;
    const int op[3] = {0, 0, 0};
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const LatDesc& d = t.d[j];
        double v[3] = {0, 0, 0};
        for (int b = threadIdx.x; b < d.red_blocks; b += blockDim.x)
            for (int k = 0; k < 3; ++k) v[k] += d.partials[b * PARTIAL_STRIDE + k];
        block_reduce<3>(v, op, sm);
        if (threadIdx.x == 0) {
            d.rec->sum_m = v[0];
            d.rec->sum_dr = v[1];
            d.rec->mass_now = v[2];
            d.rec->proj = v[0] > 0.0 ? (v[1] + (v[2] - d.rec->mass0)) / v[0] : 0.0;
        }
    }
}

// Per-cell corrected density and raw momentum change, shared by the second reduction and
// the apply pass so both see identical values.
// Per-cell arithmetic runs in the lattice's arithmetic type R (FP32 for FP32/FP16 storage,
// FP64 for FP64 storage); only the lattice-wide sums are FP64.
template <typename R>
struct CellCorr {
    R m, rhop, djx_raw, djy_raw;
};
template <typename R>
struct CorrK {
    R gmax, proj, beta_rho, beta_u, eps;  // proj = (sum drho_raw + M - M0) / sum m; eps: the band
};
template <typename R>
__device__ __forceinline__ CorrK<R> corr_constants(const DevRecord* rec, double beta_rho, double beta_u,
                                                   double eps) {
    CorrK<R> k;
    k.gmax = R(rec->gmax);
    k.proj = R(rec->proj);
    k.beta_rho = R(beta_rho);
    k.beta_u = R(beta_u);
    k.eps = R(eps);
    return k;
}
// The cell's fields, loaded together (one memory round trip per cell).
template <typename R>
struct CellIn {
    R r, jx, jy, g, rh, ux, uy;  // rho, j, |grad rho|, network rho^, u^
};
template <typename R>
__device__ __forceinline__ CellIn<R> cell_in(long long c, const R* rho, const R* jx, const R* jy, const R* g,
                                             const R* out3, long long N) {
    return CellIn<R>{rho[c], jx[c], jy[c], g[c], out3[c], out3[N + c], out3[2 * N + c]};
}
template <typename R>
__device__ __forceinline__ CellCorr<R> cell_corr(const CellIn<R>& in, const CorrK<R>& k) {
    CellCorr<R> q;
    q.m = in.g / k.gmax;
    if (!(q.m > k.eps)) {   // outside the interface band: unchanged (the network is not read)
        q.m = R(0);
        q.rhop = in.r;
        q.djx_raw = q.djy_raw = R(0);
        return q;
    }
    const R dr = k.beta_rho * q.m * (in.rh - in.r) - q.m * k.proj;
    q.rhop = in.r + dr;
    q.djx_raw = k.beta_u * q.m * (q.rhop * in.ux - in.jx);
    q.djy_raw = k.beta_u * q.m * (q.rhop * in.uy - in.jy);
    return q;
}
template <typename R>
__device__ __forceinline__ CellCorr<R> cell_corr(long long c, const R* rho, const R* jx, const R* jy, const R* g,
                                                 const R* out3, long long N, const CorrK<R>& k) {
    return cell_corr(cell_in(c, rho, jx, jy, g, out3, N), k);
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_corr_sums2(TableView t) {
    __shared__ double sm[3 * 32];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    const int op[3] = {0, 0, 1};
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        const long long N = (long long)d.nx * d.ny;
        SumAcc<R> s_jx, s_jy;  // sum djx_raw, sum djy_raw
        bool reject = false;
        if (d.rec->sum_m > 0.0) {
            const CorrK<R> k = corr_constants<R>(d.rec, d.beta_rho, d.beta_u, d.mask_eps);
            const long long step = (long long)d.red_blocks * RB_THREADS;
            for (long long c0 = (long long)m.lb * RB_THREADS + threadIdx.x; c0 < N; c0 += 2 * step) {
                // two cells' loads together, then the cells in walk order
                const bool v1 = c0 + step < N;
                const CellIn<R> in0 = cell_in(c0, static_cast<const R*>(d.rho), static_cast<const R*>(d.jx),
                                              static_cast<const R*>(d.jy), static_cast<const R*>(d.g),
                                              static_cast<const R*>(d.out3), N);
                CellIn<R> in1{};
                if (v1)
                    in1 = cell_in(c0 + step, static_cast<const R*>(d.rho), static_cast<const R*>(d.jx),
                                  static_cast<const R*>(d.jy), static_cast<const R*>(d.g),
                                  static_cast<const R*>(d.out3), N);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (u == 1 && !v1) break;
                    const CellCorr<R> q = cell_corr(u == 0 ? in0 : in1, k);
                    s_jx.add(q.djx_raw);
                    s_jy.add(q.djy_raw);
                    const bool ok = q.rhop > R(0) && isfinite(q.rhop) && isfinite(q.djx_raw) && isfinite(q.djy_raw);
                    reject = reject || !ok;
                }
            }
        }
        double v[3];
        if constexpr (std::is_same<R, float>::value) {
            float hi[3] = {s_jx.hi, s_jy.hi, reject ? 1.0f : 0.0f}, lo[3] = {s_jx.lo, s_jy.lo, 0.0f};
            block_reduce_ff<3>(hi, lo, op, reinterpret_cast<float*>(sm), v);
        } else {
            v[0] = s_jx.value(), v[1] = s_jy.value(), v[2] = reject ? 1.0 : 0.0;
            block_reduce<3>(v, op, sm);
        }
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) d.partials[m.lb * PARTIAL_STRIDE + k] = v[k];
    }
}

__global__ void __launch_bounds__(RB_THREADS) k_corr_final2(TableView t) {
    __shared__ double sm[3 * 32];
    const int n = t.hdr->n;
    const int op[3] = {0, 0, 1};
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const LatDesc& d = t.d[j];
        double v[3] = {0, 0, 0};
        for (int b = threadIdx.x; b < d.red_blocks; b += blockDim.x) {
            v[0] += d.partials[b * PARTIAL_STRIDE + 0];
            v[1] += d.partials[b * PARTIAL_STRIDE + 1];
            v[2] = fmax(v[2], d.partials[b * PARTIAL_STRIDE + 2]);
        }
        block_reduce<3>(v, op, sm);
        if (threadIdx.x == 0) {
            DevRecord* rec = d.rec;
            rec->sum_jx = v[0];
            rec->sum_jy = v[1];
            rec->mjx = rec->sum_m > 0.0 ? v[0] / rec->sum_m : 0.0;
            rec->mjy = rec->sum_m > 0.0 ? v[1] / rec->sum_m : 0.0;
            rec->reject = v[2] > 0.0 ? 1 : 0;
            if (v[2] > 0.0) {
                if (rec->status == PL_OK) rec->status = PL_ERR_NONPHYSICAL;
            } else if (rec->sum_m > 0.0) {
                rec->applied += 1;
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void feq9(R rho, R ux, R uy, R (&fe)[9]) {
    const R usq = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R cu = R(cx(i)) * ux + R(cy(i)) * uy;
        fe[i] = wq<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - usq);
    }
}

// The correction changes the populations of a corrected cell by f_i^eq(rho', u') - f_i^eq(rho, u).
// FP16-offset storage applies it to the stored offsets directly (the references, and with
// them the decoding, stay as they are): every offset is rounded stochastically (the
// conversion with random bits), the rest offset taking the cell's corrected mass minus the
// rounded moving offsets, so small changes are realised on average instead of being rounded
// away and rounding adds no bias to the mass or the momentum.
template <int MODE>
__global__ void __launch_bounds__(RB_THREADS, MODE == PL_F16_OFFSET ? 4 : 1) k_corr_apply(TableView t, int parity) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    const uint32_t seq = t.seq[parity];
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        const DevRecord* rec = d.rec;
        if (rec->reject || !(rec->sum_m > 0.0)) continue;
        const long long N = (long long)d.nx * d.ny;
        const R* rho = static_cast<const R*>(d.rho);
        const R* jx = static_cast<const R*>(d.jx);
        const R* jy = static_cast<const R*>(d.jy);
        const R* g = static_cast<const R*>(d.g);
        const R* out3 = static_cast<const R*>(d.out3);
        S* f = static_cast<S*>(d.pops[d.phase ^ parity]);
        const R sjx = R(rec->mjx), sjy = R(rec->mjy);
        const CorrK<R> k = corr_constants<R>(rec, d.beta_rho, d.beta_u, d.mask_eps);
        for (CellIt it((long long)m.lb * RB_THREADS + threadIdx.x, (long long)d.red_blocks * RB_THREADS, d.nx); it.c < N;
             it.next(d.nx)) {
            const long long c = it.c;
            const long long o = it.pop_offset(d.pitch);
            // every load of the cell first, independent of each other
            const CellIn<R> in = cell_in(c, rho, jx, jy, g, out3, N);
            S fs[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) fs[i] = f[i * d.plane + o];
            const CellCorr<R> q = cell_corr(in, k);
            if (!(q.m > R(0))) continue;
            const R djx = q.djx_raw - q.m * sjx, djy = q.djy_raw - q.m * sjy;
            const R r = in.r, jxc = in.jx, jyc = in.jy;
            R fn[9], fo[9];
            feq9<R>(q.rhop, (jxc + djx) / q.rhop, (jyc + djy) / q.rhop, fn);
            feq9<R>(r, jxc / r, jyc / r, fo);
            // the moment fields follow the corrected state, from the values stored (the cells
            // left alone keep theirs), so the metric pass after the correction need not
            // recompute them
            if constexpr (MODE == PL_F16_OFFSET) {
                float hn[9], hs[9], tt[9];
                float res = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) hn[i] = fmaf(F16_SCALE, fn[i] - fo[i], __half2float(fs[i]));
                uint32_t st = fmix32(__float_as_uint(hn[0]) ^ ((uint32_t)c * 0x9E3779B1u) ^
                                     ((seq - d.seq0) * 0x27D4EB2Fu));
#pragma unroll
                for (int i = 1; i < 9; i += 2) {
                    st = st * 1664525u + 1013904223u;
                    const uint32_t q2 = rs_pack(hn[i], hn[i + 1], st);
                    const __half qa = __ushort_as_half((unsigned short)(q2 & 0xFFFFu));
                    const __half qb = __ushort_as_half((unsigned short)(q2 >> 16));
                    hs[i] = __half2float(qa);
                    hs[i + 1] = __half2float(qb);
                    res += (hs[i] - hn[i]) + (hs[i + 1] - hn[i + 1]);
                    f[i * d.plane + o] = qa;
                    f[(i + 1) * d.plane + o] = qb;
                }
                st = st * 1664525u + 1013904223u;
                const __half q0 = __ushort_as_half((unsigned short)(rs_pack(hn[0] - res, 0.0f, st) & 0xFFFFu));
                f[o] = q0;
                hs[0] = __half2float(q0);
#pragma unroll
                for (int i = 0; i < 9; ++i) hs[i] *= F16_UNSCALE;
                f16_refs(f, d.plane, d.pitch, d.nx, d.ny, it.x, it.y, tt);
                put_moments_f16(d, c, hs, tt);
            } else {
                R P[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const S v = encode<MODE>(decode<MODE>(fs[i]) + (fn[i] - fo[i]));
                    f[i * d.plane + o] = v;
                    P[i] = decode<MODE>(v);
                }
                put_moments_p<R>(d, c, P);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The correction's interface band (lattices with mask_eps > 0): the cells whose mask
// m = g / G_max is above mask_eps, compacted per lattice into d.band (block by block in the
// fixed reduction partition, within a block thread by thread in walk order: deterministic), so
// that the network is evaluated on the band only.  The mask is formed as in cell_corr.

// A thread's band cells (or their count when out == nullptr) in its walk order.
template <typename R>
__device__ __forceinline__ unsigned band_walk(const LatDesc& d, int lb, int* out) {
    const R* g = static_cast<const R*>(d.g);
    const R gmax = R(d.rec->gmax), eps = R(d.mask_eps);
    const long long N = (long long)d.nx * d.ny;
    unsigned n = 0;
    for (long long c = (long long)lb * RB_THREADS + threadIdx.x; c < N; c += (long long)d.red_blocks * RB_THREADS) {
        const R m = gmax > R(0) ? g[c] / gmax : R(0);
        if (m > eps) {
            if (out) out[n] = (int)c;
            ++n;
        }
    }
    return n;
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_band_count(TableView t) {
    __shared__ double sm[32];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    const int op[1] = {0};
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        if (!(d.mask_eps > 0.0)) continue;
        double v[1] = {(double)band_walk<R>(d, m.lb, nullptr)};
        block_reduce<1>(v, op, sm);
        if (threadIdx.x == 0) d.partials[m.lb * PARTIAL_STRIDE + 0] = v[0];
    }
}

// One thread per lattice: each block's first band position (slot 1) and the band's size.
__global__ void k_band_scan(TableView t) {
    const int n = t.hdr->n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const LatDesc& d = t.d[j];
        if (!(d.mask_eps > 0.0)) {
            d.rec->band_n = -1;
            continue;
        }
        double off = 0.0;
        for (int b = 0; b < d.red_blocks; ++b) {
            d.partials[b * PARTIAL_STRIDE + 1] = off;
            off += d.partials[b * PARTIAL_STRIDE + 0];
        }
        d.rec->band_n = (int)off;
    }
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_band_write(TableView t) {
    __shared__ unsigned scan[RB_THREADS];
    const int n = t.hdr->n, total = t.hdr->total_blocks;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const BlkMap m = map_blk(t, n, vb);
        const LatDesc& d = t.d[m.j];
        if (!(d.mask_eps > 0.0)) continue;
        // exclusive scan of the per-thread counts (Hillis-Steele in shared memory)
        const unsigned cnt = band_walk<R>(d, m.lb, nullptr);
        scan[threadIdx.x] = cnt;
        __syncthreads();
        for (int off = 1; off < RB_THREADS; off <<= 1) {
            const unsigned add = threadIdx.x >= off ? scan[threadIdx.x - off] : 0u;
            __syncthreads();
            scan[threadIdx.x] += add;
            __syncthreads();
        }
        const long long first = (long long)d.partials[m.lb * PARTIAL_STRIDE + 1] + scan[threadIdx.x] - cnt;
        __syncthreads();
        band_walk<R>(d, m.lb, d.band + first);
    }
}

template <int MODE>
static cudaError_t correction_t(const TableView& t, int parity, int mlp_mode, int n_in, const float* w32,
                                const uint16_t* wbf16, cudaStream_t s) {
    using R = typename Traits<MODE>::R;
    k_moments<MODE><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);  // rho, j (and the stencil input)
    k_grad_tab<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_final_metrics_tab<<<RED_GRID, RB_THREADS, 0, s>>>(t, 0);
    // the interface band of lattices with mask_eps > 0 (the network then runs on it only)
    k_band_count<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_band_scan<<<(RED_GRID + 127) / 128, 128, 0, s>>>(t);
    k_band_write<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    note_launches(3);
    cudaError_t e = launch_mlp_tab(t, MODE, mlp_mode, n_in, w32, wbf16, s, 1);
    if (e != cudaSuccess) return e;
    k_corr_sums1<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_corr_final1<<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_corr_sums2<R><<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_corr_final2<<<RED_GRID, RB_THREADS, 0, s>>>(t);
    k_corr_apply<MODE><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);
    note_launches(8);
    return cudaGetLastError();
}

cudaError_t launch_correction_tab(const TableView& t, int storage, int parity, int mlp_mode, int n_in,
                                  const float* w32, const uint16_t* wbf16, cudaStream_t s) {
    switch (storage) {
        case PL_F64: return correction_t<PL_F64>(t, parity, mlp_mode, n_in, w32, wbf16, s);
        case PL_F32: return correction_t<PL_F32>(t, parity, mlp_mode, n_in, w32, wbf16, s);
        case PL_F16_OFFSET: return correction_t<PL_F16_OFFSET>(t, parity, mlp_mode, n_in, w32, wbf16, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_train_fields_tab(const TableView& t, int storage, int parity, cudaStream_t s) {
    switch (storage) {
        case PL_F64:
            k_moments<PL_F64><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);
            k_grad_tab<double><<<RED_GRID, RB_THREADS, 0, s>>>(t);
            break;
        case PL_F32:
            k_moments<PL_F32><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);
            k_grad_tab<float><<<RED_GRID, RB_THREADS, 0, s>>>(t);
            break;
        case PL_F16_OFFSET:
            k_moments<PL_F16_OFFSET><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity);
            k_grad_tab<float><<<RED_GRID, RB_THREADS, 0, s>>>(t);
            break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_moments_tab(const TableView& t, int storage, int parity, cudaStream_t s) {
    switch (storage) {
        case PL_F64: k_moments<PL_F64><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity); break;
        case PL_F32: k_moments<PL_F32><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity); break;
        case PL_F16_OFFSET: k_moments<PL_F16_OFFSET><<<RED_GRID, RB_THREADS, 0, s>>>(t, parity); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Allocation-free metrics (pl_metrics_noalloc).  Some callers cannot allocate device memory
// at all: code running where cudaMalloc is forbidden or unavailable (inside another
// library's allocator or its stream-ordered pool callbacks, or a host that must not grow
// its device footprint after start-up), or code that owns no scratch buffer to lend.  For
// them this variant of the metric reduction keeps its scratch - the density field, the
// per-block partials and the record - in one file-scope __device__ array instead of in a
// caller buffer.  Every GPU that loads the library holds the array until the process exits.

constexpr long long NOALLOC_MAX_CELLS = 1ll << 20;  // largest lattice: 1,048,576 cells
constexpr int NOALLOC_BLOCKS = 1024;                 // reduction blocks (partials capacity)
constexpr size_t NOALLOC_RHO_BYTES = (size_t)NOALLOC_MAX_CELLS * sizeof(double);
constexpr size_t NOALLOC_PART_BYTES = (size_t)NOALLOC_BLOCKS * PARTIAL_STRIDE * sizeof(double);
constexpr size_t NOALLOC_BYTES = NOALLOC_RHO_BYTES + NOALLOC_PART_BYTES + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Density of every cell from populations in the library's layout, into a dense array.
template <int MODE>
__global__ void k_density_noalloc(const typename Traits<MODE>::S* __restrict__ f, int nx, int ny, int pitch,
                                  long long plane, typename Traits<MODE>::R* __restrict__ rho) {
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        if constexpr (MODE == PL_F16_OFFSET) {
            float h[9], tt[9];
            f16_cell(f, plane, pitch, nx, ny, x, y, h, tt);
            rho[c] = sum9(tt) + sum9(h);
        } else {
            const long long o = (long long)y * pitch + x;
            R P[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) P[i] = decode<MODE>(f[i * plane + o]);
            rho[c] = ((P[0] + P[1]) + (P[2] + P[3])) + ((P[4] + P[5]) + (P[6] + P[7])) + P[8];
        }
    }
}

template <int MODE>
static void metrics_noalloc_t(const void* pops, int nx, int ny, int pitch, double threshold,
                              unsigned char* scratch, DevRecord* rec, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    long long nb = (N + RB_THREADS - 1) / RB_THREADS;
    if (nb > NOALLOC_BLOCKS) nb = NOALLOC_BLOCKS;
    R* rho = reinterpret_cast<R*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + NOALLOC_RHO_BYTES);
    k_density_noalloc<MODE><<<(int)nb, RB_THREADS, 0, s>>>(static_cast<const S*>(pops), nx, ny, pitch,
                                                           (long long)pitch * ny, rho);
    k_grad_reduce<R><<<(int)nb, RB_THREADS, 0, s>>>(rho, nx, ny, nullptr, threshold, partials);
    k_final_metrics<<<1, RB_THREADS, 0, s>>>(partials, (int)nb, rec, 0);
    note_launches(3);
}
static_assert(sizeof(DevRecord) <= 256, "record slot of the static scratch");

}  // namespace pl

extern "C" PL_API int pl_metrics_noalloc(const void* dev_pops, int32_t nx, int32_t ny, int32_t pitch, int32_t storage,
                                         double rho_ref, double threshold, void* stream, pl_metric_record* out) {
    using namespace pl;
    if (!dev_pops || !out || nx < 1 || ny < 1 || pitch < nx || !std::isfinite(rho_ref) || !std::isfinite(threshold))
        return PL_ERR_INVALID_ARG;
    if (storage != PL_F64 && storage != PL_F32 && storage != PL_F16_OFFSET) return PL_ERR_INVALID_ARG;
    const size_t esize = storage == PL_F64 ? 8 : (storage == PL_F32 ? 4 : 2);
    if ((uintptr_t)dev_pops % esize) return PL_ERR_INVALID_ARG;
    if ((long long)nx * ny > NOALLOC_MAX_CELLS) {
        std::fprintf(stderr, "pl_metrics_noalloc: lattice of %lld cells exceeds the %lld-cell maximum of the "
                             "static scratch\n", (long long)nx * ny, NOALLOC_MAX_CELLS);
        return PL_ERR_BUDGET;
    }
    // In host code g_noalloc_scratch names a host-side stand-in, not device memory: the
    // array's address on the current device is looked up on every call (a cheap query), so
    // no address outlives the context it belongs to (a cudaDeviceReset reloads the module).
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return PL_ERR_CUDA;
    }
    unsigned char* scratch = static_cast<unsigned char*>(p);
    DevRecord* rec = reinterpret_cast<DevRecord*>(scratch + NOALLOC_RHO_BYTES + NOALLOC_PART_BYTES);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(rec, 0, sizeof(DevRecord), s);  // the record starts at zero on every call
    if (e == cudaSuccess) {
        switch (storage) {
            case PL_F64: metrics_noalloc_t<PL_F64>(dev_pops, nx, ny, pitch, threshold, scratch, rec, s); break;
            case PL_F32: metrics_noalloc_t<PL_F32>(dev_pops, nx, ny, pitch, threshold, scratch, rec, s); break;
            default: metrics_noalloc_t<PL_F16_OFFSET>(dev_pops, nx, ny, pitch, threshold, scratch, rec, s); break;
        }
        e = cudaGetLastError();
    }
    DevRecord r;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, rec, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return PL_ERR_CUDA;
    }
    const double N = (double)nx * (double)ny;
    std::memset(out, 0, sizeof(*out));
    out->mass = r.mass;
    out->count = r.count;
    out->W = (double)r.count / N;
    out->G_max = r.gmax;
    out->delta_rho = r.rho_max - r.rho_min;
    out->W_eff = r.gmax > 0.0 ? r.sum_g / (r.gmax * N) : 0.0;
    out->E_int = r.sum_g2;
    out->rho_max = r.rho_max;
    out->rho_min = r.rho_min;
    out->sum_g = r.sum_g;
    out->sum_g2 = r.sum_g2;
    out->R_eq = out->rho_in = out->rho_out = out->p_in = out->p_out = out->dP = NAN;
    out->mass0 = NAN;
    return PL_OK;
}
