// Lattice kernels of the time step (arXiv 2504.10539 Sec. II-A, Eq. 1) and
// of the initial state (Sec. III-A).
//
// Storage: structure of arrays, 9 planes of nx*ny populations (x fastest),
// two buffers (two-lattice "push": read the post-streaming state of buffer
// src, write the next post-streaming state into buffer 1-src).  Reads of a
// step never alias its writes, so a CTA may recompute its neighbours' density
// from their populations without racing with them: the result is identical
// whatever the launch order.
//
// Fused step kernel, one pass over HBM per step:
//   - a CTA owns a strip of TX-2 columns and TY rows; thread t handles column
//     x0-1+t (the two edge threads only supply the pseudopotential halo);
//   - it walks its rows bottom to top ("rolling window"), keeping three rows of
//     psi in a 4-slot shared-memory ring, so each cell's populations are read
//     from HBM once and only the two halo rows/columns are read twice (from L2);
//   - per owned cell: rho, psi, the Shan-Chen force from the 3x3 psi stencil,
//     the force-shifted equilibrium, BGK relaxation, and the push to the 8
//     neighbours with periodic wrap, all in registers.
#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

template <int MODE>
__global__ void __launch_bounds__(256) k_step(const typename Traits<MODE>::S* __restrict__ fin,
                                              typename Traits<MODE>::S* __restrict__ fout, int nx, int ny,
                                              long long plane, int ty, typename Traits<MODE>::R G,
                                              typename Traits<MODE>::R tau, typename Traits<MODE>::R omega,
                                              typename Traits<MODE>::R rho0, typename Traits<MODE>::R rho_ref) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* psi_s = reinterpret_cast<R*>(smem_raw);  // [4][TX]

    const int TX = blockDim.x;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * (TX - 2);
    const int xg = x0 - 1 + t;
    const int xc = wrapi(xg, nx);
    const bool owner = (t >= 1) && (t <= TX - 2) && (xg < nx);
    const int xm = xc == 0 ? nx - 1 : xc - 1;
    const int xp = xc == nx - 1 ? 0 : xc + 1;
    const int y0 = blockIdx.y * ty;
    const int rows = min(ty, ny - y0);
    const R inv_rho0 = R(1) / rho0;

    R off[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) off[i] = wq<R>(i) * rho_ref;

    R Pn[9], Pc[9], Pp[9];
    R rho_p = R(0);
    {
        const S* b = fin + (long long)wrapi(y0 - 1, ny) * nx + xc;
#pragma unroll
        for (int i = 0; i < 9; ++i) Pn[i] = decode<MODE>(b[i * plane], off[i]);
    }
    for (int k = 0; k <= rows + 1; ++k) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Pc[i] = Pn[i];
        if (k <= rows) {  // prefetch the next row while this one is processed
            int rn = y0 + k;
            if (rn >= ny) rn -= ny;
            const S* b = fin + (long long)rn * nx + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i) Pn[i] = decode<MODE>(b[i * plane], off[i]);
        }
        R rho_c = ((Pc[0] + Pc[1]) + (Pc[2] + Pc[3])) + ((Pc[4] + Pc[5]) + (Pc[6] + Pc[7])) + Pc[8];
        psi_s[(k & 3) * TX + t] = psi_of(rho_c, rho0, inv_rho0);
        __syncthreads();
        if (k >= 2 && owner) {
            const int y = y0 + k - 2;
            const R* sm = psi_s + ((k - 2) & 3) * TX;  // row y-1
            const R* s0 = psi_s + ((k - 1) & 3) * TX;  // row y
            const R* sp = psi_s + (k & 3) * TX;        // row y+1
            const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
            const R sx = w1 * (s0[t + 1] - s0[t - 1]) + w2 * ((sp[t + 1] - sp[t - 1]) + (sm[t + 1] - sm[t - 1]));
            const R sy = w1 * (sp[t] - sm[t]) + w2 * ((sp[t + 1] + sp[t - 1]) - (sm[t + 1] + sm[t - 1]));
            const R gpsi = -G * s0[t];
            const R Fx = gpsi * sx, Fy = gpsi * sy;

            const R rho = rho_p;
            const R inv = R(1) / rho;
            const R jx = (Pp[1] - Pp[3]) + (Pp[5] - Pp[6]) + (Pp[8] - Pp[7]);
            const R jy = (Pp[2] - Pp[4]) + (Pp[5] + Pp[6]) - (Pp[7] + Pp[8]);
            const R ux = (jx + tau * Fx) * inv;  // u + tau F / rho
            const R uy = (jy + tau * Fy) * inv;
            const R usq = R(1.5) * (ux * ux + uy * uy);
            R out[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R cu = R(cx(i)) * ux + R(cy(i)) * uy;
                const R feq = wq<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - usq);
                out[i] = Pp[i] + omega * (feq - Pp[i]);
            }
            const long long ry = (long long)y * nx;
            const long long rm = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
            const long long rp = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
            fout[0 * plane + ry + xc] = encode<MODE>(out[0], off[0]);
            fout[1 * plane + ry + xp] = encode<MODE>(out[1], off[1]);
            fout[2 * plane + rp + xc] = encode<MODE>(out[2], off[2]);
            fout[3 * plane + ry + xm] = encode<MODE>(out[3], off[3]);
            fout[4 * plane + rm + xc] = encode<MODE>(out[4], off[4]);
            fout[5 * plane + rp + xp] = encode<MODE>(out[5], off[5]);
            fout[6 * plane + rp + xm] = encode<MODE>(out[6], off[6]);
            fout[7 * plane + rm + xm] = encode<MODE>(out[7], off[7]);
            fout[8 * plane + rm + xp] = encode<MODE>(out[8], off[8]);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) Pp[i] = Pc[i];
        rho_p = rho_c;
    }
}

StepTiling default_tiling(int nx, int ny) {
    StepTiling t;
    int tx = ((nx + 2 + 31) / 32) * 32;
    t.tx = tx > 128 ? 128 : tx;
    t.ty = ny < 32 ? ny : 32;
    (void)ny;
    return t;
}

template <int MODE>
static cudaError_t launch_step_t(const LatticeView& v, const PhysParams& p, int src, StepTiling tl, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    dim3 grid((v.nx + tl.tx - 3) / (tl.tx - 2), (v.ny + tl.ty - 1) / tl.ty);
    size_t smem = 4 * tl.tx * sizeof(R);
    k_step<MODE><<<grid, tl.tx, smem, s>>>(static_cast<const S*>(v.pops[src]), static_cast<S*>(v.pops[1 - src]), v.nx,
                                           v.ny, v.plane, tl.ty, R(p.G), R(p.tau), R(1.0 / p.tau), R(p.rho0),
                                           R(p.rho_ref));
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_step(const LatticeView& v, const PhysParams& p, int src, StepTiling tl, cudaStream_t s) {
    if (tl.tx < 32 || tl.tx > 256 || (tl.tx & 31) || tl.ty < 1) return cudaErrorInvalidValue;
    switch (v.storage) {
        case PL_F64: return launch_step_t<PL_F64>(v, p, src, tl, s);
        case PL_F32: return launch_step_t<PL_F32>(v, p, src, tl, s);
        case PL_F16_OFFSET: return launch_step_t<PL_F16_OFFSET>(v, p, src, tl, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Initial state (Sec. III-A): tanh droplet profile(s), counter-based noise, f_i = w_i rho.

__device__ __forceinline__ double min_image(double d, double n) {
    double a = fabs(fmod(d, n));
    return a > 0.5 * n ? n - a : a;
}

template <int MODE>
__global__ void k_init_droplets(typename Traits<MODE>::S* __restrict__ f, int nx, int ny, long long plane,
                                const pl_droplet* __restrict__ d, int n, double rho_in, double rho_out, double width,
                                double noise_amp, uint64_t seed, double rho_ref) {
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        double best = 0.0;
        for (int k = 0; k < n; ++k) {
            const double dx = min_image((double)x - d[k].cx, (double)nx);
            const double dy = min_image((double)y - d[k].cy, (double)ny);
            const double d2 = dx * dx + dy * dy;
            const double cut = d[k].r + 20.0 * width;  // tanh((d-r)/width) == 1 exactly beyond this
            if (d2 > cut * cut) continue;
            const double phi = 0.5 * (1.0 - tanh((sqrt(d2) - d[k].r) / width));
            best = phi > best ? phi : best;
        }
        const double rho = rho_out + (rho_in - rho_out) * best + noise_amp * (2.0 * uniform01_at(seed, (uint64_t)c) - 1.0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double fi = wq<double>(i) * rho;
            f[i * plane + c] = encode<MODE>(R(fi), R(wq<double>(i) * rho_ref));
        }
    }
}

template <int MODE>
__global__ void k_init_from_rho(typename Traits<MODE>::S* __restrict__ f, long long N, long long plane,
                                const double* __restrict__ rho, double rho_ref) {
    using R = typename Traits<MODE>::R;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * plane + c] = encode<MODE>(R(wq<double>(i) * rho[c]), R(wq<double>(i) * rho_ref));
    }
}

// FP64 exchange format <-> storage, one plane per launch (plane index `i`).
template <int MODE>
__global__ void k_plane_convert(typename Traits<MODE>::S* __restrict__ f, long long N, long long plane, int i,
                                double* __restrict__ buf, int to_f64, double rho_ref) {
    using R = typename Traits<MODE>::R;
    const R off = R(wq<double>(i) * rho_ref);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        if (to_f64) buf[c] = (double)decode<MODE>(f[i * plane + c], off);
        else f[i * plane + c] = encode<MODE>(R(buf[c]), off);
    }
}

static int grid_for(long long N) {
    long long b = (N + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

cudaError_t launch_init_droplets(const LatticeView& v, const PhysParams& p, int cur, int n, double rho_in,
                                 double rho_out, double width, double noise_amp, uint64_t seed, cudaStream_t s) {
    const long long N = (long long)v.nx * v.ny;
    switch (v.storage) {
        case PL_F64:
            k_init_droplets<PL_F64><<<grid_for(N), 256, 0, s>>>(static_cast<double*>(v.pops[cur]), v.nx, v.ny, v.plane,
                                                               v.droplets, n, rho_in, rho_out, width, noise_amp, seed,
                                                               p.rho_ref);
            break;
        case PL_F32:
            k_init_droplets<PL_F32><<<grid_for(N), 256, 0, s>>>(static_cast<float*>(v.pops[cur]), v.nx, v.ny, v.plane,
                                                               v.droplets, n, rho_in, rho_out, width, noise_amp, seed,
                                                               p.rho_ref);
            break;
        case PL_F16_OFFSET:
            k_init_droplets<PL_F16_OFFSET><<<grid_for(N), 256, 0, s>>>(static_cast<__half*>(v.pops[cur]), v.nx, v.ny,
                                                                      v.plane, v.droplets, n, rho_in, rho_out, width,
                                                                      noise_amp, seed, p.rho_ref);
            break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init_from_rho(const LatticeView& v, const PhysParams& p, int cur, const double* d_rho,
                                 cudaStream_t s) {
    const long long N = (long long)v.nx * v.ny;
    switch (v.storage) {
        case PL_F64:
            k_init_from_rho<PL_F64><<<grid_for(N), 256, 0, s>>>(static_cast<double*>(v.pops[cur]), N, v.plane, d_rho, p.rho_ref);
            break;
        case PL_F32:
            k_init_from_rho<PL_F32><<<grid_for(N), 256, 0, s>>>(static_cast<float*>(v.pops[cur]), N, v.plane, d_rho, p.rho_ref);
            break;
        case PL_F16_OFFSET:
            k_init_from_rho<PL_F16_OFFSET><<<grid_for(N), 256, 0, s>>>(static_cast<__half*>(v.pops[cur]), N, v.plane,
                                                                      d_rho, p.rho_ref);
            break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_state_convert(const LatticeView& v, const PhysParams& p, int cur, double* d_buf, int i, int to_f64,
                                 cudaStream_t s) {
    const long long N = (long long)v.nx * v.ny;
    switch (v.storage) {
        case PL_F64:
            k_plane_convert<PL_F64><<<grid_for(N), 256, 0, s>>>(static_cast<double*>(v.pops[cur]), N, v.plane, i, d_buf,
                                                               to_f64, p.rho_ref);
            break;
        case PL_F32:
            k_plane_convert<PL_F32><<<grid_for(N), 256, 0, s>>>(static_cast<float*>(v.pops[cur]), N, v.plane, i, d_buf,
                                                               to_f64, p.rho_ref);
            break;
        case PL_F16_OFFSET:
            k_plane_convert<PL_F16_OFFSET><<<grid_for(N), 256, 0, s>>>(static_cast<__half*>(v.pops[cur]), N, v.plane, i,
                                                                      d_buf, to_f64, p.rho_ref);
            break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pl
