// Interface metrics (arXiv 2504.10539 Sec. II-D Eqs. 9-13, discretised in
// Sec. IV-E Eqs. 14-16), the mass, and the Laplace measurement.
//
// Two-level deterministic reductions: a fixed grid of RB blocks accumulates
// per-thread FP64 partial sums / extrema over a fixed grid-stride assignment
// of cells, reduces them by a fixed warp-shuffle tree into one partial per
// block, and a one-block kernel folds the partials in block order.  The result
// does not depend on scheduling, so repeated runs are bit-identical.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

constexpr int RB_THREADS = 256;
constexpr int RB_MAX_BLOCKS = 1024;
constexpr int PARTIAL_STRIDE = 8;  // doubles per block partial

int reduction_blocks(const LatticeView& v) {
    long long N = (long long)v.nx * v.ny;
    long long b = (N + RB_THREADS - 1) / RB_THREADS;
    if (b > v.max_blocks) b = v.max_blocks;
    if (b > RB_MAX_BLOCKS) b = RB_MAX_BLOCKS;
    return (int)(b < 1 ? 1 : b);
}

// rho = sum_i f_i and j = sum_i f_i c_i per cell, from the decoded stored state.
template <int MODE>
__global__ void k_moments(const typename Traits<MODE>::S* __restrict__ f, int nx, int pitch, long long N,
                          long long plane, typename Traits<MODE>::R rho_ref, typename Traits<MODE>::R* __restrict__ rho,
                          typename Traits<MODE>::R* __restrict__ jx, typename Traits<MODE>::R* __restrict__ jy) {
    using R = typename Traits<MODE>::R;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long o = (c / nx) * pitch + c % nx;
        R P[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = decode<MODE>(f[i * plane + o], wq<R>(i) * rho_ref);
        rho[c] = ((P[0] + P[1]) + (P[2] + P[3])) + ((P[4] + P[5]) + (P[6] + P[7])) + P[8];
        jx[c] = (P[1] - P[3]) + (P[5] - P[6]) + (P[8] - P[7]);
        jy[c] = (P[2] - P[4]) + (P[5] + P[6]) - (P[7] + P[8]);
    }
}

// Eq. 16 gradient magnitude (central differences, periodic, dx = dy = 1), stored
// to g, and the per-block partials {sum rho, max g, sum g, sum g^2, max rho, min rho, count(g > thr)}.
template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_grad_reduce(const R* __restrict__ rho, int nx, int ny,
                                                            R* __restrict__ g, double threshold,
                                                            double* __restrict__ partials) {
    __shared__ double sm[7 * 32];
    const long long N = (long long)nx * ny;
    double v[7] = {0.0, 0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    const int op[7] = {0, 1, 0, 0, 1, 2, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const long long row = c - x;
        const R gx = (rho[row + (x == nx - 1 ? 0 : x + 1)] - rho[row + (x == 0 ? nx - 1 : x - 1)]) / R(2);
        const R gy = (rho[(long long)(y == ny - 1 ? 0 : y + 1) * nx + x] - rho[(long long)(y == 0 ? ny - 1 : y - 1) * nx + x]) / R(2);
        const R gm = sqrt(gx * gx + gy * gy);
        if (g) g[c] = gm;
        const double r = (double)rho[c], gd = (double)gm;
        v[0] += r;
        v[1] = fmax(v[1], gd);
        v[2] += gd;
        v[3] += gd * gd;
        v[4] = fmax(v[4], r);
        v[5] = fmin(v[5], r);
        v[6] += gd > threshold ? 1.0 : 0.0;
    }
    block_reduce<7>(v, op, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) partials[blockIdx.x * PARTIAL_STRIDE + k] = v[k];
}

// Fold the block partials into the lattice record.
__global__ void __launch_bounds__(RB_THREADS) k_final_metrics(const double* __restrict__ partials, int nb,
                                                              DevRecord* rec, int set_mass0) {
    __shared__ double sm[7 * 32];
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
        if (set_mass0) rec->mass0 = v[0];
    }
}

// Laplace measurement about (cx, cy) (build-defined estimator, Sec. III-A set-up):
// R_eq = sqrt((M - N rho_out) / (pi (rho_in - rho_out))); inner cells d < R_eq/2,
// outer cells d > R_eq + 4 width; means of rho and of p = rho/3 + G psi^2/6.
__device__ __forceinline__ double min_image_d(double d, double n) {
    double a = fabs(fmod(d, n));
    return a > 0.5 * n ? n - a : a;
}

__device__ __forceinline__ double laplace_req(const DevRecord* rec, long long N) {
    return sqrt((rec->mass - (double)N * rec->rho_out) / (3.14159265358979323846 * (rec->rho_in - rec->rho_out)));
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_laplace_region(const R* __restrict__ rho, int nx, int ny, double cx,
                                                               double cy, double width, double G, double rho0,
                                                               const DevRecord* __restrict__ rec,
                                                               double* __restrict__ partials) {
    __shared__ double sm[6 * 32];
    const long long N = (long long)nx * ny;
    const double Req = laplace_req(rec, N);
    double v[6] = {0, 0, 0, 0, 0, 0};  // inner: sum rho, sum p, n; outer: sum rho, sum p, n
    const int op[6] = {0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const double dx = min_image_d((double)x - cx, (double)nx), dy = min_image_d((double)y - cy, (double)ny);
        const double d = sqrt(dx * dx + dy * dy);
        const double r = (double)rho[c];
        const double ps = -rho0 * expm1(-r / rho0);
        const double p = r / 3.0 + G * ps * ps / 6.0;
        if (d < 0.5 * Req) { v[0] += r; v[1] += p; v[2] += 1.0; }
        if (d > Req + 4.0 * width) { v[3] += r; v[4] += p; v[5] += 1.0; }
    }
    block_reduce<6>(v, op, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) partials[blockIdx.x * PARTIAL_STRIDE + k] = v[k];
}

__global__ void __launch_bounds__(RB_THREADS) k_laplace_final(const double* __restrict__ partials, int nb, long long N,
                                                              DevRecord* rec) {
    __shared__ double sm[6 * 32];
    double v[6] = {0, 0, 0, 0, 0, 0};
    const int op[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < 6; ++k) v[k] += partials[b * PARTIAL_STRIDE + k];
    block_reduce<6>(v, op, sm);
    if (threadIdx.x == 0) {
        rec->R_eq = laplace_req(rec, N);
        rec->rho_in = v[2] > 0 ? v[0] / v[2] : NAN;
        rec->p_in = v[2] > 0 ? v[1] / v[2] : NAN;
        rec->rho_out = v[5] > 0 ? v[3] / v[5] : NAN;
        rec->p_out = v[5] > 0 ? v[4] / v[5] : NAN;
    }
}

template <int MODE>
static cudaError_t metrics_t(const LatticeView& v, const PhysParams& p, int cur, int has_centre, double cx, double cy,
                             double width, int set_mass0, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const long long N = (long long)v.nx * v.ny;
    const int nb = reduction_blocks(v);
    R* rho = static_cast<R*>(v.rho);
    k_moments<MODE><<<nb, RB_THREADS, 0, s>>>(static_cast<const S*>(v.pops[cur]), v.nx, v.pitch, N, v.plane,
                                              R(p.rho_ref), rho, static_cast<R*>(v.jx), static_cast<R*>(v.jy));
    k_grad_reduce<R><<<nb, RB_THREADS, 0, s>>>(rho, v.nx, v.ny, static_cast<R*>(v.g), p.threshold, v.partials);
    k_final_metrics<<<1, RB_THREADS, 0, s>>>(v.partials, nb, v.rec, set_mass0);
    if (has_centre) {
        for (int it = 0; it < 2; ++it) {
            k_laplace_region<R><<<nb, RB_THREADS, 0, s>>>(rho, v.nx, v.ny, cx, cy, width, p.G, p.rho0, v.rec, v.partials);
            k_laplace_final<<<1, RB_THREADS, 0, s>>>(v.partials, nb, N, v.rec);
        }
    }
    note_launches(has_centre ? 7 : 3);
    return cudaGetLastError();
}

cudaError_t launch_metrics(const LatticeView& v, const PhysParams& p, int cur, int has_centre, double cx, double cy,
                           double width, int set_mass0, cudaStream_t s) {
    switch (v.storage) {
        case PL_F64: return metrics_t<PL_F64>(v, p, cur, has_centre, cx, cy, width, set_mass0, s);
        case PL_F32: return metrics_t<PL_F32>(v, p, cur, has_centre, cx, cy, width, set_mass0, s);
        case PL_F16_OFFSET: return metrics_t<PL_F16_OFFSET>(v, p, cur, has_centre, cx, cy, width, set_mass0, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Interface correction reductions and apply (Sec. II-C step 3; the operator is the build's
// reading, the paper gives none):
//   m = g / G_max; drho_raw = beta_rho m (rho^ - rho)
//   drho = drho_raw - m (sum drho_raw + (M - M0)) / sum m;  rho' = rho + drho
//   dj_raw = beta_u m (rho' u^ - j); dj = dj_raw - m sum dj_raw / sum m;  u' = (j + dj) / rho'
//   f_i += f_i^eq(rho', u') - f_i^eq(rho, u) on cells with m > 0.

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_corr_sums1(const R* __restrict__ rho, const R* __restrict__ g,
                                                           const R* __restrict__ out3, long long N, double beta_rho,
                                                           const DevRecord* __restrict__ rec,
                                                           double* __restrict__ partials) {
    __shared__ double sm[3 * 32];
    const double gmax = rec->gmax;
    double v[3] = {0, 0, 0};  // sum m, sum drho_raw, sum rho
    const int op[3] = {0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double r = (double)rho[c];
        const double m = gmax > 0.0 ? (double)g[c] / gmax : 0.0;
        v[0] += m;
        v[1] += beta_rho * m * ((double)out3[c] - r);
        v[2] += r;
    }
    block_reduce<3>(v, op, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partials[blockIdx.x * PARTIAL_STRIDE + k] = v[k];
}

__global__ void __launch_bounds__(RB_THREADS) k_corr_final1(const double* __restrict__ partials, int nb, DevRecord* rec) {
    __shared__ double sm[3 * 32];
    double v[3] = {0, 0, 0};
    const int op[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < 3; ++k) v[k] += partials[b * PARTIAL_STRIDE + k];
    block_reduce<3>(v, op, sm);
    if (threadIdx.x == 0) {
        rec->sum_m = v[0];
        rec->sum_dr = v[1];
        rec->mass_now = v[2];
    }
}

// Per-cell corrected density and raw momentum change, shared by the second
// reduction and the apply pass so both see identical values.
struct CellCorr {
    double m, rhop, djx_raw, djy_raw;
};
template <typename R>
__device__ __forceinline__ CellCorr cell_corr(long long c, const R* rho, const R* jx, const R* jy, const R* g,
                                              const R* out3, long long N, double beta_rho, double beta_u,
                                              const DevRecord* rec) {
    CellCorr q;
    const double r = (double)rho[c];
    q.m = (double)g[c] / rec->gmax;
    const double dr_raw = beta_rho * q.m * ((double)out3[c] - r);
    const double dr = dr_raw - q.m * (rec->sum_dr + (rec->mass_now - rec->mass0)) / rec->sum_m;
    q.rhop = r + dr;
    q.djx_raw = beta_u * q.m * (q.rhop * (double)out3[N + c] - (double)jx[c]);
    q.djy_raw = beta_u * q.m * (q.rhop * (double)out3[2 * N + c] - (double)jy[c]);
    return q;
}

template <typename R>
__global__ void __launch_bounds__(RB_THREADS) k_corr_sums2(const R* __restrict__ rho, const R* __restrict__ jx,
                                                           const R* __restrict__ jy, const R* __restrict__ g,
                                                           const R* __restrict__ out3, long long N, double beta_rho,
                                                           double beta_u, const DevRecord* __restrict__ rec,
                                                           double* __restrict__ partials) {
    __shared__ double sm[3 * 32];
    double v[3] = {0, 0, 0};  // sum djx_raw, sum djy_raw, reject flag
    const int op[3] = {0, 0, 1};
    if (rec->sum_m > 0.0) {
        for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
            const CellCorr q = cell_corr(c, rho, jx, jy, g, out3, N, beta_rho, beta_u, rec);
            v[0] += q.djx_raw;
            v[1] += q.djy_raw;
            const bool ok = q.rhop > 0.0 && isfinite(q.rhop) && isfinite(q.djx_raw) && isfinite(q.djy_raw);
            v[2] = fmax(v[2], ok ? 0.0 : 1.0);
        }
    }
    block_reduce<3>(v, op, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partials[blockIdx.x * PARTIAL_STRIDE + k] = v[k];
}

__global__ void __launch_bounds__(RB_THREADS) k_corr_final2(const double* __restrict__ partials, int nb, DevRecord* rec) {
    __shared__ double sm[3 * 32];
    double v[3] = {0, 0, 0};
    const int op[3] = {0, 0, 1};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        v[0] += partials[b * PARTIAL_STRIDE + 0];
        v[1] += partials[b * PARTIAL_STRIDE + 1];
        v[2] = fmax(v[2], partials[b * PARTIAL_STRIDE + 2]);
    }
    block_reduce<3>(v, op, sm);
    if (threadIdx.x == 0) {
        rec->sum_jx = v[0];
        rec->sum_jy = v[1];
        rec->reject = v[2] > 0.0 ? 1 : 0;
        if (v[2] > 0.0) {
            if (rec->status == PL_OK) rec->status = PL_ERR_NONPHYSICAL;
        } else if (rec->sum_m > 0.0) {
            rec->applied += 1;
        }
    }
}

template <typename R>
__device__ __forceinline__ void feq9(double rho, double ux, double uy, double (&fe)[9]) {
    const double usq = 1.5 * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy;
        fe[i] = wq<double>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - usq);
    }
}

template <int MODE>
__global__ void k_corr_apply(typename Traits<MODE>::S* __restrict__ f, int nx, int pitch, long long plane,
                             const typename Traits<MODE>::R* __restrict__ rho, const typename Traits<MODE>::R* __restrict__ jx,
                             const typename Traits<MODE>::R* __restrict__ jy, const typename Traits<MODE>::R* __restrict__ g,
                             const typename Traits<MODE>::R* __restrict__ out3, long long N, double beta_rho,
                             double beta_u, double rho_ref, const DevRecord* __restrict__ rec) {
    using R = typename Traits<MODE>::R;
    if (rec->reject || !(rec->sum_m > 0.0)) return;
    const double sjx = rec->sum_jx / rec->sum_m, sjy = rec->sum_jy / rec->sum_m;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        if (!((double)g[c] > 0.0)) continue;
        const CellCorr q = cell_corr(c, rho, jx, jy, g, out3, N, beta_rho, beta_u, rec);
        const double djx = q.djx_raw - q.m * sjx, djy = q.djy_raw - q.m * sjy;
        const double r = (double)rho[c], jxc = (double)jx[c], jyc = (double)jy[c];
        double fn[9], fo[9];
        feq9<R>(q.rhop, (jxc + djx) / q.rhop, (jyc + djy) / q.rhop, fn);
        feq9<R>(r, jxc / r, jyc / r, fo);
        const long long o = (c / nx) * pitch + c % nx;
        if constexpr (MODE == PL_F16_OFFSET) {
            // stored offsets h_i + (f_i^eq' - f_i^eq): the moving populations rounded to
            // nearest, the rest population taking the cell's corrected stored mass minus their
            // rounded values and rounded stochastically, so that small per-cell changes
            // (below half an FP16 step) are realised on average instead of being rounded away
            float hn[9];
            float res = 0.0f;
#pragma unroll
            for (int i = 0; i < 9; ++i) hn[i] = __half2float(f[i * plane + o]) + (float)(fn[i] - fo[i]);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const __half q = __float2half_rn(hn[i]);
                res += __half2float(q) - hn[i];
                f[i * plane + o] = q;
            }
            const uint32_t rnd = fmix32(__float_as_uint(hn[0]) ^ ((uint32_t)c * 0x9E3779B1u));
            f[o] = sr_half(hn[0] - res, rnd);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R off = R(wq<double>(i) * rho_ref);
                const double fi = (double)decode<MODE>(f[i * plane + o], off);
                f[i * plane + o] = encode<MODE>(R(fi + (fn[i] - fo[i])), off);
            }
        }
    }
}

template <int MODE>
static cudaError_t correction_t(const LatticeView& v, const PhysParams& p, int cur, int mlp_mode, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const long long N = (long long)v.nx * v.ny;
    const int nb = reduction_blocks(v);
    R* rho = static_cast<R*>(v.rho);
    R* jx = static_cast<R*>(v.jx);
    R* jy = static_cast<R*>(v.jy);
    R* g = static_cast<R*>(v.g);
    R* out3 = static_cast<R*>(v.out3);
    cudaError_t e = launch_mlp_field(v, mlp_mode, s);
    if (e != cudaSuccess) return e;
    k_moments<MODE><<<nb, RB_THREADS, 0, s>>>(static_cast<const S*>(v.pops[cur]), v.nx, v.pitch, N, v.plane, R(p.rho_ref),
                                              rho, jx, jy);
    k_grad_reduce<R><<<nb, RB_THREADS, 0, s>>>(rho, v.nx, v.ny, g, p.threshold, v.partials);
    k_final_metrics<<<1, RB_THREADS, 0, s>>>(v.partials, nb, v.rec, 0);
    k_corr_sums1<R><<<nb, RB_THREADS, 0, s>>>(rho, g, out3, N, p.beta_rho, v.rec, v.partials);
    k_corr_final1<<<1, RB_THREADS, 0, s>>>(v.partials, nb, v.rec);
    k_corr_sums2<R><<<nb, RB_THREADS, 0, s>>>(rho, jx, jy, g, out3, N, p.beta_rho, p.beta_u, v.rec, v.partials);
    k_corr_final2<<<1, RB_THREADS, 0, s>>>(v.partials, nb, v.rec);
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_corr_apply<MODE><<<(int)blocks, 256, 0, s>>>(static_cast<S*>(v.pops[cur]), v.nx, v.pitch, v.plane, rho, jx, jy, g, out3, N,
                                                   p.beta_rho, p.beta_u, p.rho_ref, v.rec);
    note_launches(8);
    return cudaGetLastError();
}

cudaError_t launch_correction(const LatticeView& v, const PhysParams& p, int cur, int mlp_mode, cudaStream_t s) {
    switch (v.storage) {
        case PL_F64: return correction_t<PL_F64>(v, p, cur, mlp_mode, s);
        case PL_F32: return correction_t<PL_F32>(v, p, cur, mlp_mode, s);
        case PL_F16_OFFSET: return correction_t<PL_F16_OFFSET>(v, p, cur, mlp_mode, s);
    }
    return cudaErrorInvalidValue;
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
                                  long long plane, typename Traits<MODE>::R rho_ref,
                                  typename Traits<MODE>::R* __restrict__ rho) {
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long o = (c / nx) * pitch + c % nx;
        R P[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = decode<MODE>(f[i * plane + o], wq<R>(i) * rho_ref);
        rho[c] = ((P[0] + P[1]) + (P[2] + P[3])) + ((P[4] + P[5]) + (P[6] + P[7])) + P[8];
    }
}

template <int MODE>
static void metrics_noalloc_t(const void* pops, int nx, int ny, int pitch, double rho_ref, double threshold,
                              unsigned char* scratch, DevRecord* rec, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    long long nb = (N + RB_THREADS - 1) / RB_THREADS;
    if (nb > NOALLOC_BLOCKS) nb = NOALLOC_BLOCKS;
    R* rho = reinterpret_cast<R*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + NOALLOC_RHO_BYTES);
    k_density_noalloc<MODE><<<(int)nb, RB_THREADS, 0, s>>>(static_cast<const S*>(pops), nx, ny, pitch,
                                                           (long long)pitch * ny, R(rho_ref), rho);
    k_grad_reduce<R><<<(int)nb, RB_THREADS, 0, s>>>(rho, nx, ny, nullptr, threshold, partials);
    k_final_metrics<<<1, RB_THREADS, 0, s>>>(partials, (int)nb, rec, 0);
    note_launches(3);
}
static_assert(sizeof(DevRecord) <= 256, "record slot of the static scratch");

}  // namespace pl

namespace {
// Device address of g_noalloc_scratch, looked up once per device (with that device current).
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};
}  // namespace

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return PL_ERR_CUDA;
    }
    unsigned char* scratch;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return PL_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    }
    DevRecord* rec = reinterpret_cast<DevRecord*>(scratch + NOALLOC_RHO_BYTES + NOALLOC_PART_BYTES);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(rec, 0, sizeof(DevRecord), s);  // the record starts at zero on every call
    if (e == cudaSuccess) {
        switch (storage) {
            case PL_F64: metrics_noalloc_t<PL_F64>(dev_pops, nx, ny, pitch, rho_ref, threshold, scratch, rec, s); break;
            case PL_F32: metrics_noalloc_t<PL_F32>(dev_pops, nx, ny, pitch, rho_ref, threshold, scratch, rec, s); break;
            default: metrics_noalloc_t<PL_F16_OFFSET>(dev_pops, nx, ny, pitch, rho_ref, threshold, scratch, rec, s); break;
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
