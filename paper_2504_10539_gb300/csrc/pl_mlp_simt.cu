// Correction network on CUDA cores (FP64 or FP32), arXiv 2504.10539 Sec. II-B
// Eq. 2 and Sec. III-B: N(x, y) = (rho^, u^_x, u^_y), 2 -> 64 -> 128 -> 128 -> 64 -> 3,
// tanh on the hidden layers, linear output.  Input: the cell centre mapped to
// [-1, 1] (x^ = 2 (x + 0.5) / nx - 1); with n_in = 11 (a stencil variant the paper does
// not have) also the density of the cell and its 8 neighbours, velocity order, periodic.
//
// A block takes 32 cells at a time (a 128-cell tile of lattice j is four 32-cell parts), its
// four warps splitting each layer's outputs among them (warp w computes outputs w n/4 ..
// (w + 1) n/4 - 1 of its layer for all 32 cells, lane = cell): a small lattice's cells spread
// over four times as many SMs as tiles, each with four warps, which the FP64 form, bound by the
// FP64 rate and latency of the SMs it occupies, needs.  Every output is one thread's sum over
// its inputs in order, so the split changes no result.  Activations live in shared memory,
// feature-major ([feature][cell]) so that a warp's accesses are consecutive; each thread
// accumulates 16 outputs at a time in registers while the weights (the same for the whole
// warp) are broadcast from the read-only cache.
#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

cudaError_t launch_mlp_tc(const TableView& t, const float* w32, const uint16_t* wbf16, int n_in, int use_band,
                          cudaStream_t s);

constexpr int MLP_CELLS = 32;                      // cells per block at a time (one per lane)
constexpr int MLP_SLICES = 4;                      // warps per block: output slices of each layer
constexpr int MLP_THREADS = MLP_CELLS * MLP_SLICES;
constexpr int MLP_PARTS = MLP_TILE / MLP_CELLS;    // parts of a 128-cell tile, one block each
constexpr int MLP_CHUNK = 16;
constexpr int MLP_GRID = 152 * 8;

template <typename R>
__device__ __forceinline__ R act_tanh(R z);
template <>
__device__ __forceinline__ float act_tanh<float>(float z) { return tanhf(z); }
template <>
__device__ __forceinline__ double act_tanh<double>(double z) { return tanh(z); }

// One dense layer in -> out, this thread's slice of the outputs for its cell:
// dst[o] = act(sum_k W[o][k] src[k] + b[o]).
template <typename R, bool TANH>
__device__ __forceinline__ void dense(const float* __restrict__ W, const float* __restrict__ b, int nin, int nout,
                                      const R* src, R* dst, int cell, int slice) {
    const int per = (nout + MLP_SLICES - 1) / MLP_SLICES;
    const int lo = slice * per, hi = min(nout, lo + per);
    for (int o0 = lo; o0 < hi; o0 += MLP_CHUNK) {
        R acc[MLP_CHUNK];
#pragma unroll
        for (int j = 0; j < MLP_CHUNK; ++j) acc[j] = (o0 + j < hi) ? R(__ldg(b + o0 + j)) : R(0);
        for (int k = 0; k < nin; ++k) {
            const R a = src[k * MLP_CELLS + cell];
#pragma unroll
            for (int j = 0; j < MLP_CHUNK; ++j)
                if (o0 + j < hi) acc[j] += R(__ldg(W + (o0 + j) * nin + k)) * a;
        }
#pragma unroll
        for (int j = 0; j < MLP_CHUNK; ++j)
            if (o0 + j < hi) dst[(o0 + j) * MLP_CELLS + cell] = TANH ? act_tanh<R>(acc[j]) : acc[j];
    }
    __syncthreads();  // the next layer reads every output of this one
}

__device__ __forceinline__ int find_tile_s(const long long* __restrict__ pre, int n, long long v) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename R>
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_simt(const float* __restrict__ w, TableView tab, int n_in) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* bufA = reinterpret_cast<R*>(smem_raw);     // [128][MLP_CELLS]
    R* bufB = bufA + 128 * MLP_CELLS;              // [128][MLP_CELLS]
    const int cell = threadIdx.x % MLP_CELLS, slice = threadIdx.x / MLP_CELLS;
    const int nlat = tab.hdr->n;
    const long long parts = MLP_PARTS * tab.hdr->total_tiles;
    // blob offsets
    const float* W1 = w;
    const float* b1 = W1 + 64 * n_in;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 128 * 64;
    const float* W3 = b2 + 128;
    const float* b3 = W3 + 128 * 128;
    const float* W4 = b3 + 128;
    const float* b4 = W4 + 64 * 128;
    const float* W5 = b4 + 64;
    const float* b5 = W5 + 3 * 64;
    for (long long vh = blockIdx.x; vh < parts; vh += gridDim.x) {
        const long long tile = vh / MLP_PARTS;
        const int j = find_tile_s(tab.tile_pre, nlat, tile);
        const LatDesc& d = tab.d[j];
        const int nx = d.nx, ny = d.ny;
        const long long N = (long long)nx * ny;
        R* out3 = static_cast<R*>(d.out3);
        const long long c = (tile - tab.tile_pre[j]) * MLP_TILE + (vh % MLP_PARTS) * MLP_CELLS + cell;
        const long long cc = c < N ? c : N - 1;
        if (slice == 0) {
            // 32-bit division (a lattice holds fewer than 2^31 cells)
            const int y = (int)((uint32_t)cc / (uint32_t)nx), x = (int)((uint32_t)cc - (uint32_t)y * (uint32_t)nx);
            bufA[0 * MLP_CELLS + cell] = R(2) * (R(x) + R(0.5)) / R(nx) - R(1);
            bufA[1 * MLP_CELLS + cell] = R(2) * (R(y) + R(0.5)) / R(ny) - R(1);
            if (n_in == 11) {
                const R* rho = static_cast<const R*>(d.rho);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    int xn = x + cx(i), yn = y + cy(i);
                    xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
                    yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
                    bufA[(2 + i) * MLP_CELLS + cell] = rho[(long long)yn * nx + xn];
                }
            }
        }
        __syncthreads();
        dense<R, true>(W1, b1, n_in, 64, bufA, bufB, cell, slice);
        dense<R, true>(W2, b2, 64, 128, bufB, bufA, cell, slice);
        dense<R, true>(W3, b3, 128, 128, bufA, bufB, cell, slice);
        dense<R, true>(W4, b4, 128, 64, bufB, bufA, cell, slice);
        dense<R, false>(W5, b5, 64, 3, bufA, bufB, cell, slice);
        if (slice == 0 && c < N) {
            out3[c] = bufB[0 * MLP_CELLS + cell];
            out3[N + c] = bufB[1 * MLP_CELLS + cell];
            out3[2 * N + c] = bufB[2 * MLP_CELLS + cell];
        }
        __syncthreads();  // the next part rewrites the buffers
    }
}

template <typename R>
static cudaError_t mlp_simt_t(const TableView& t, const float* w32, int n_in, cudaStream_t s) {
    const size_t smem = 2 * 128 * MLP_CELLS * sizeof(R);
    static bool attr_set = false;  // per process and instantiation (one device)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_simt<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_mlp_simt<R><<<MLP_GRID, MLP_THREADS, smem, s>>>(w32, t, n_in);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tab(const TableView& t, int storage, int mlp_mode, int n_in, const float* w32,
                           const uint16_t* wbf16, cudaStream_t s, int use_band) {
    if (n_in != 2 && n_in != 11) return cudaErrorInvalidValue;
    // The output element type follows the lattice's scratch type: double for FP64 storage.
    if (storage == PL_F64) {
        if (mlp_mode != PL_MLP_F64) return cudaErrorInvalidValue;
        return mlp_simt_t<double>(t, w32, n_in, s);
    }
    if (mlp_mode == PL_MLP_BF16) return launch_mlp_tc(t, w32, wbf16, n_in, use_band, s);  // (CUDA cores: every cell)
    if (mlp_mode != PL_MLP_F32) return cudaErrorInvalidValue;
    return mlp_simt_t<float>(t, w32, n_in, s);
}

// Seeded weights (Sec. III-B gives the architecture; "seed-initialised" fixes no
// distribution, so the fan-in uniform is used): entry k of the FP32 blob, in blob order
// (layer by layer, W[out][in] row-major, then b), is (2 U(seed, k) - 1) / sqrt(fan_in), U the
// SplitMix64 uniform of output k (top 53 bits), rounded to FP32 to nearest.  All arithmetic
// in FP64 with correctly rounded sqrt and division, so the blob is the same bits on any host.
__global__ void k_init_weights(float* __restrict__ w32, int n_in, uint64_t seed) {
    const int dims[6] = {n_in, 64, 128, 128, 64, 3};
    int ends[5];
    int e = 0;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        e += dims[l + 1] * dims[l] + dims[l + 1];
        ends[l] = e;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < e; k += gridDim.x * blockDim.x) {
        int l = 0;
        while (k >= ends[l]) ++l;
        const double t = 2.0 * uniform01_at(seed, (uint64_t)k) - 1.0;
        w32[k] = __double2float_rn(t * (1.0 / sqrt((double)dims[l])));
    }
}

cudaError_t launch_init_weights(float* w32, int n_in, uint64_t seed, cudaStream_t s) {
    if (n_in != 2 && n_in != 11) return cudaErrorInvalidValue;
    k_init_weights<<<64, 256, 0, s>>>(w32, n_in, seed);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pl
