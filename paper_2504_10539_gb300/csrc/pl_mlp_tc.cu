// Correction network on tcgen05 tensor cores (sm_103a): BF16 operands in shared
// memory, FP32 accumulators in tensor memory (TMEM).
//
// N(x, y) -> (rho^, u^_x, u^_y) (arXiv 2504.10539 Sec. II-B Eq. 2, Sec. III-B):
// 2 -> 64 -> 128 -> 128 -> 64 -> 3, tanh on the hidden layers, linear output.
//   layer 1 (2 -> 64)     : FP32 FMA per cell, tanh, rounded to BF16 (A operand of layer 2)
//   layers 2, 3, 4        : tcgen05.mma kind::f16, M = 128 cells, N = 128/128/64, K = 64/128/128,
//                           plus one K = 16 step that adds the bias (ones x [b_hi, b_lo]);
//                           D in TMEM; epilogue tcgen05.ld -> tanh -> BF16 -> smem
//   layer 5 (64 -> 3)     : FP32 FMA on the FP32 tanh outputs of layer 4
//
// CTA = 4 warpgroups (16 warps, all TMEM columns); each warpgroup runs its own 128-cell
// tile pipeline with its own operand buffer, 128 TMEM columns and mbarrier, so the
// warpgroups' tanh epilogues overlap each other's MMAs and hide each other's latencies.
// One 32 KB operand buffer per warpgroup suffices: a layer's epilogue writes the next
// operand only after the layer's MMA has completed (its mbarrier), i.e. after the MMA has
// read the buffer.  Thread t of a warpgroup owns cell row t of the tile
// (TMEM lane t: warp w of the group reads lanes 32*(w%4)..+31).  The weights are
// loaded once per CTA by bulk async copies (the grid is persistent, one CTA per SM).
//
// Operand layout (no swizzle, K-major): 8x8 BF16 "core matrices" of 128 contiguous
// bytes (8 rows of 16 bytes).  An R x K operand is stored core-matrix (kb, rb) at
// byte ((kb * R/8) + rb) * 128, so core matrices adjacent in R are 128 B apart
// (stride byte offset) and those adjacent in K are R/8 * 128 B apart (leading
// byte offset).  One MMA consumes K = 16, i.e. two core matrices along K.
//
// Every wait on an mbarrier is bounded by %globaltimer; on expiry the warpgroup
// records an error, stops issuing work, waits (bounded) for its MMAs in flight,
// and the CTA frees its TMEM before returning.
#include <cuda_bf16.h>

#include "pl_device.cuh"
#include "pl_kernels.h"
#include "pl_tcgen05.cuh"

namespace pl {

namespace tc {

constexpr int M = 128;           // cells per tile
constexpr int NWG = 4;           // tile pipelines per CTA
constexpr int THREADS = 128 * NWG;
constexpr int TMEM_COLS = 128 * NWG;

// shared memory map (bytes).  A buffers first, weight images next, FP32 params
// last; the allocation is the full 227 KB so that every address an MMA can form
// from these bases stays inside it.
constexpr int A_BYTES = M * 128 * 2;                 // 128 rows x 128 BF16 = 32 KB
constexpr int OFF_A = 0;                             // one operand buffer per WG
constexpr int OFF_W2 = OFF_A + NWG * A_BYTES;        // 128 x 64  BF16 = 16 KB
constexpr int OFF_W3 = OFF_W2 + 128 * 64 * 2;        // 128 x 128 BF16 = 32 KB
constexpr int OFF_W4 = OFF_W3 + 128 * 128 * 2;       // 64 x 128  BF16 = 16 KB
constexpr int WB_ELEMS = (128 + 128 + 64) * 16;      // bias blocks of layers 2-4: N x 16 BF16
constexpr int OFF_WB = OFF_W4 + 64 * 128 * 2;        // (bias split hi + lo in K columns 0 and 1)
constexpr int OFF_ONES = OFF_WB + WB_ELEMS * 2;      // 128 x 16 BF16 A operand: columns 0, 1 = 1
constexpr int OFF_P = OFF_ONES + M * 16 * 2;         // FP32 parameters
// FP32 parameters of layers 1 and 5 (the biases of layers 2-4 are in the MMA): W1 as 64 rows of
// n_in inputs, packed (n_in = 2) or padded to 12 (n_in = 11, 16-byte rows); b1; W5; b5
constexpr int P_W1 = 0, P_B1 = 768, P_W5 = 832, P_B5 = 1024, P_N = 1028;
constexpr int OFF_BAR = (OFF_P + P_N * 4 + 15) / 16 * 16;
constexpr int OFF_TMEM_SLOT = OFF_BAR + 8 * (1 + NWG);
constexpr int SMEM_USED = OFF_TMEM_SLOT + 16;
constexpr int SMEM_ALLOC = 227 * 1024;
static_assert(OFF_BAR % 8 == 0, "mbarrier alignment");
static_assert(SMEM_USED <= SMEM_ALLOC, "shared memory");

constexpr int W_IMG_ELEMS = 128 * 64 + 128 * 128 + 64 * 128 + WB_ELEMS;   // BF16 image in global memory

// Blob offsets (FP32 master weights, row-major W[out][in]).
struct BlobOff {
    int W1, B1, W2, B2, W3, B3, W4, B4, W5, B5;
};
__host__ __device__ constexpr BlobOff blob_off(int n_in) {
    return BlobOff{0,
                   64 * n_in,
                   64 * n_in + 64,
                   64 * n_in + 64 + 8192,
                   64 * n_in + 64 + 8192 + 128,
                   64 * n_in + 64 + 8192 + 128 + 16384,
                   64 * n_in + 64 + 8192 + 128 + 16384 + 128,
                   64 * n_in + 64 + 8192 + 128 + 16384 + 128 + 8192,
                   64 * n_in + 64 + 8192 + 128 + 16384 + 128 + 8192 + 64,
                   64 * n_in + 64 + 8192 + 128 + 16384 + 128 + 8192 + 64 + 192};
}

// Issue D[128 x N] = A[128 x K] * W[N x K]^T + bias as K/16 + 1 MMAs: the bias enters the
// FP32 accumulator through one more K = 16 step, a block of ones (columns 0 and 1) times the
// bias split into BF16 high and low parts (b = b_hi + b_lo to 2^-16 relative).
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, uint32_t a_base, uint32_t w_base, int N, int K,
                                            uint32_t ones_base, uint32_t bias_base) {
    const uint32_t idesc = idesc_bf16(M, N);
    const uint32_t a_lbo = (M / 8) * 128, w_lbo = (N / 8) * 128;
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t a = smem_desc(a_base + ks * 2 * a_lbo, a_lbo, 128);
        const uint64_t b = smem_desc(w_base + ks * 2 * w_lbo, w_lbo, 128);
        mma_bf16(d_tmem, a, b, idesc, ks > 0 ? 1u : 0u);
    }
    mma_bf16(d_tmem, smem_desc(ones_base, a_lbo, 128), smem_desc(bias_base, w_lbo, 128), idesc, 1u);
}

}  // namespace tc

size_t bf16_weight_elems() { return tc::W_IMG_ELEMS; }

// FP32 blob -> BF16 (round to nearest even) images of W2, W3, W4 in the core-matrix
// layout above: element (n, k) of an N x K matrix at ((k/8) * N/8 + n/8) * 64 + (n%8) * 8 + k%8;
// then the bias blocks of layers 2, 3, 4 (N x 16, same layout): column 0 = bf16(b),
// column 1 = bf16(b - bf16(b)), the other columns 0.
__global__ void k_convert_weights_bf16(const float* __restrict__ w32, uint16_t* __restrict__ img, int n_in) {
    constexpr int NW = 8192 + 16384 + 8192;
    const tc::BlobOff bo = tc::blob_off(n_in);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tc::W_IMG_ELEMS; e += gridDim.x * blockDim.x) {
        int N, K, base, loc;
        float v;
        if (e < NW) {
            int src;
            if (e < 8192) { N = 128; K = 64; src = bo.W2; base = 0; loc = e; }
            else if (e < 8192 + 16384) { N = 128; K = 128; src = bo.W3; base = 8192; loc = e - 8192; }
            else { N = 64; K = 128; src = bo.W4; base = 8192 + 16384; loc = e - 8192 - 16384; }
            v = w32[src + (loc / K) * K + loc % K];
        } else {
            int src;
            K = 16;
            if (e < NW + 2048) { N = 128; src = bo.B2; base = NW; loc = e - NW; }
            else if (e < NW + 4096) { N = 128; src = bo.B3; base = NW + 2048; loc = e - NW - 2048; }
            else { N = 64; src = bo.B4; base = NW + 4096; loc = e - NW - 4096; }
            const float b = w32[src + loc / 16], hi = __bfloat162float(__float2bfloat16_rn(b));
            v = loc % 16 == 0 ? b : (loc % 16 == 1 ? b - hi : 0.0f);
        }
        const int n = loc / K, k = loc % K;
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        img[base + ((k >> 3) * (N >> 3) + (n >> 3)) * 64 + (n & 7) * 8 + (k & 7)] = *reinterpret_cast<uint16_t*>(&b);
    }
}

cudaError_t launch_convert_weights_bf16(const float* w32, uint16_t* wbf16, int n_in, cudaStream_t s) {
    if (n_in != 2 && n_in != 11) return cudaErrorInvalidValue;
    k_convert_weights_bf16<<<32, 256, 0, s>>>(w32, wbf16, n_in);
    note_launches(1);
    return cudaGetLastError();
}

// The lattice j with pre[j] <= v < pre[j+1], searched in [lo, n) (pre[lo] <= v).
__device__ __forceinline__ int find_tile(const long long* __restrict__ pre, int lo, int n, long long v) {
    int hi = n;  // pre[lo] <= v < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Persistent over the table's 128-cell tiles (tile v of the table belongs to the lattice j
// with tile_pre[j] <= v < tile_pre[j+1]; tiles never straddle lattices).
// NIN = 2 (the paper's inputs) or 11 (with the density stencil): one instantiation each, so
// that the paper's form keeps its own register allocation.
template <int NIN>
__global__ void __launch_bounds__(tc::THREADS, 1)
    k_mlp_tc(const uint16_t* __restrict__ wimg, const float* __restrict__ w32, TableView tab, int use_band) {
    constexpr int n_in = NIN;
    using namespace tc;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, warp = tid >> 5;
    const int nlat = tab.hdr->n;
    const long long ntiles = tab.hdr->total_tiles;
    if ((long long)blockIdx.x * NWG >= ntiles) return;  // no tile for this CTA: skip set-up
    float* P = reinterpret_cast<float*>(sm + OFF_P);
    const uint32_t bar_w = saddr(sm + OFF_BAR);
    const uint32_t bar_mma = saddr(sm + OFF_BAR + 8 * (1 + wg));
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM_SLOT);

    if (tid == 0) {
        mbar_init(bar_w, 1);
        for (int g = 0; g < NWG; ++g) mbar_init(saddr(sm + OFF_BAR + 8 * (1 + g)), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // small FP32 parameters
    const BlobOff bo = blob_off(n_in);
    if constexpr (NIN == 2) {
        for (int k = tid; k < 128; k += THREADS) P[P_W1 + k] = w32[bo.W1 + k];
    } else {
        for (int k = tid; k < 64 * 12; k += THREADS) P[P_W1 + k] = k % 12 < 11 ? w32[bo.W1 + (k / 12) * 11 + k % 12] : 0.0f;
    }
    for (int k = tid; k < 64; k += THREADS) P[P_B1 + k] = w32[bo.B1 + k];
    for (int k = tid; k < 192; k += THREADS) P[P_W5 + k] = w32[bo.W5 + k];
    for (int k = tid; k < 3; k += THREADS) P[P_B5 + k] = w32[bo.B5 + k];
    // the ones block (A operand of the bias step): element (m, k) at
    // ((k/8) * M/8 + m/8) * 64 + (m%8) * 8 + k%8, 1 in columns 0 and 1
    {
        uint16_t* ones = reinterpret_cast<uint16_t*>(sm + OFF_ONES);
        for (int e = tid; e < M * 16; e += THREADS) {
            const int m = e / 16, k = e % 16;
            ones[((k >> 3) * (M / 8) + (m >> 3)) * 64 + (m & 7) * 8 + (k & 7)] = k < 2 ? 0x3F80u : 0u;  // BF16 1.0
        }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) {
        // weight images: one bulk async copy per matrix onto the mbarrier
        const uint32_t bytes = W_IMG_ELEMS * 2;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w), "r"(bytes) : "memory");
        const uint8_t* src = reinterpret_cast<const uint8_t*>(wimg);
        const uint32_t dst[4] = {saddr(sm + OFF_W2), saddr(sm + OFF_W3), saddr(sm + OFF_W4), saddr(sm + OFF_WB)};
        const uint32_t len[4] = {128 * 64 * 2, 128 * 128 * 2, 64 * 128 * 2, WB_ELEMS * 2};
        uint32_t off = 0;
        for (int k = 0; k < 4; ++k) {
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             dst[k]),
                         "l"(src + off), "r"(len[k]), "r"(bar_w)
                         : "memory");
            off += len[k];
        }
    }
    bool ok = __syncthreads_and(mbar_wait(bar_w, 0)) != 0;

    uint8_t* AX = sm + OFF_A + wg * A_BYTES;
    const uint32_t ax = saddr(AX);
    const uint32_t d_tmem = tmem + wg * 128;                               // this WG's columns
    const uint32_t my_lane_tmem = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + wg * 128;
    uint32_t phase = 0;
    int pending = 0;  // MMA batches committed but not yet waited for

    DevRecord* last_rec = nullptr;
    // The lattice of the current tile and what the tile loop reads of it.  A warpgroup's tiles
    // rise, so the lookup is redone only when a tile leaves the current lattice, and then
    // searched from that lattice on (the search's dependent loads are paid once per lattice).
    int lj = 0;
    long long t_lo = 0, t_hi = -1;  // tile_pre[lj], tile_pre[lj + 1]
    const LatDesc* ldp = nullptr;
    int nx = 1, ny = 1;
    long long N = 1, nb = 0;
    float* out3 = nullptr;
    bool banded = false;
    for (long long tile = (long long)blockIdx.x * NWG + wg; ok && tile < ntiles; tile += (long long)gridDim.x * NWG) {
        if (tile >= t_hi) {
            lj = find_tile(tab.tile_pre, lj, nlat, tile);
            t_lo = tab.tile_pre[lj];
            t_hi = tab.tile_pre[lj + 1];
            ldp = &tab.d[lj];
            nx = ldp->nx;
            ny = ldp->ny;
            N = (long long)nx * ny;
            out3 = static_cast<float*>(ldp->out3);
            last_rec = ldp->rec;
            banded = use_band && ldp->mask_eps > 0.0;
            nb = banded ? ldp->rec->band_n : 0;
        }
        const LatDesc& ld = *ldp;
        // the tile's cells: consecutive cells, or (an interface band) consecutive band entries;
        // a lattice's band fills its first tiles, the others have no work (uniform per warpgroup)
        const long long pos = (tile - t_lo) * M + t;
        long long cc;
        bool valid;
        if (banded) {
            if ((tile - t_lo) * M >= nb) continue;
            valid = pos < nb;
            cc = ld.band[valid ? pos : nb - 1];
        } else {
            valid = pos < N;
            cc = valid ? pos : N - 1;
        }
        // 32-bit division (a lattice holds fewer than 2^31 cells)
        const int y = (int)((uint32_t)cc / (uint32_t)nx), x = (int)((uint32_t)cc - (uint32_t)y * (uint32_t)nx);
        const float xh = 2.0f * ((float)x + 0.5f) / (float)nx - 1.0f;
        const float yh = 2.0f * ((float)y + 0.5f) / (float)ny - 1.0f;

        // ---- layer 1 on FMA: A1 (128 x 64) into AX
        if constexpr (NIN == 11) {
            // the density of the cell and its 8 neighbours (periodic), velocity order
            const float* rho = static_cast<const float*>(ld.rho);
            float in[11];
            in[0] = xh;
            in[1] = yh;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                int xn = x + cx(i), yn = y + cy(i);
                xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
                yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
                in[2 + i] = rho[(long long)yn * nx + xn];
            }
#pragma unroll 1
            for (int k0 = 0; k0 < 64; k0 += 8) {
                const float4* b4 = reinterpret_cast<const float4*>(P + P_B1 + k0);
                const float4 bA = b4[0], bB = b4[1];
                const float bias[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
                float h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4* w4 = reinterpret_cast<const float4*>(P + P_W1 + (k0 + j) * 12);
                    const float4 a = w4[0], b = w4[1], c = w4[2];
                    float z = bias[j];
                    z = fmaf(a.x, in[0], z);
                    z = fmaf(a.y, in[1], z);
                    z = fmaf(a.z, in[2], z);
                    z = fmaf(a.w, in[3], z);
                    z = fmaf(b.x, in[4], z);
                    z = fmaf(b.y, in[5], z);
                    z = fmaf(b.z, in[6], z);
                    z = fmaf(b.w, in[7], z);
                    z = fmaf(c.x, in[8], z);
                    z = fmaf(c.y, in[9], z);
                    z = fmaf(c.z, in[10], z);
                    h[j] = tanh_fast(z);
                }
                store8(AX, t, k0, h);
            }
        } else
#pragma unroll
        for (int k0 = 0; k0 < 64; k0 += 8) {
            // parameters as 16-byte shared loads: W1 rows (o, o+1) and biases (o..o+3)
            const float4* w4 = reinterpret_cast<const float4*>(P + P_W1 + 2 * k0);
            const float4* b4 = reinterpret_cast<const float4*>(P + P_B1 + k0);
            const float4 bA = b4[0], bB = b4[1];
            const float bias[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {   // features j, j + 1 as one pair: W1 x^ + (W1 y^ + b)
                const float4 w = w4[j >> 1];
                const float2 z = fma2(make_float2(w.x, w.z), bc2(xh),
                                      fma2(make_float2(w.y, w.w), bc2(yh), make_float2(bias[j], bias[j + 1])));
                h[j] = tanh_fast(z.x);
                h[j + 1] = tanh_fast(z.y);
            }
            store8(AX, t, k0, h);
        }
        // ---- layers 2..4: MMA, then epilogue
        // layer 5: per output two packed partial sums (features = 0 / 1 mod 2, and j mod 4 < 2 or
        // not), added at the end: short dependency chains
        float2 oa[3], ob[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            oa[k] = make_float2(P[P_B5 + k], 0.0f);
            ob[k] = bc2(0.0f);
        }
#pragma unroll 1
        for (int layer = 2; layer <= 4 && ok; ++layer) {
            fence_async_smem();
            tc_before_sync();
            wg_bar(wg);
            if (t == 0) {
                tc_after_sync();
                const uint32_t ones = saddr(sm + OFF_ONES), wb = saddr(sm + OFF_WB);
                if (layer == 2) issue_layer(d_tmem, ax, saddr(sm + OFF_W2), 128, 64, ones, wb);
                else if (layer == 3) issue_layer(d_tmem, ax, saddr(sm + OFF_W3), 128, 128, ones, wb + 128 * 16 * 2);
                else issue_layer(d_tmem, ax, saddr(sm + OFF_W4), 64, 128, ones, wb + 256 * 16 * 2);
                mma_commit(bar_mma);
            }
            pending = 1;
            ok = wg_all(wg, mbar_wait(bar_mma, phase));
            if (!ok) break;
            pending = 0;
            phase ^= 1;
            tc_after_sync();
            const int nout = layer == 4 ? 64 : 128;
            uint8_t* dst = AX;  // the layer's MMA has completed: its operand buffer is free
#pragma unroll 1
            for (int c0 = 0; c0 < nout; c0 += 32) {
                float v[32];
                tmem_ld32(my_lane_tmem + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = tanh_fast(v[j]);  // the bias is in the accumulator
                if (layer < 4) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) store8(dst, t, c0 + 8 * q, v + 8 * q);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float2 va = make_float2(v[4 * q], v[4 * q + 1]), vb = make_float2(v[4 * q + 2], v[4 * q + 3]);
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float4 a = reinterpret_cast<const float4*>(P + P_W5 + k * 64 + c0)[q];
                            oa[k] = fma2(make_float2(a.x, a.y), va, oa[k]);
                            ob[k] = fma2(make_float2(a.z, a.w), vb, ob[k]);
                        }
                    }
                }
            }
        }
        if (!ok) break;
        if (valid) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float2 s2 = add2(oa[k], ob[k]);
                out3[k * N + cc] = s2.x + s2.y;
            }
        }
    }
    if (!ok) {
        if (t == 0 && last_rec) atomicCAS(&last_rec->status, PL_OK, PL_ERR_TIMEOUT);
        if (pending) (void)mbar_wait(bar_mma, phase);  // let MMAs in flight finish before TMEM is freed
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives on;
// the wait gives up after limit_ns and the kernel reports PL_ERR_TIMEOUT in *status.
__global__ void k_selftest_wait(int* status, long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = tc::saddr(&bar);
    tc::mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *status = tc::mbar_wait(b, 0, limit_ns) ? PL_OK : PL_ERR_TIMEOUT;
}

cudaError_t launch_selftest_wait(int* d_status, long long limit_ns, cudaStream_t s) {
    k_selftest_wait<<<1, 1, 0, s>>>(d_status, limit_ns);
    note_launches(1);
    return cudaGetLastError();
}

template <int NIN>
static cudaError_t launch_mlp_tc_t(const TableView& t, const float* w32, const uint16_t* wbf16, int use_band,
                                   cudaStream_t s) {
    static int sms = 0;
    if (!sms) {
        cudaError_t e =
            cudaFuncSetAttribute(k_mlp_tc<NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_ALLOC);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    // persistent: one CTA per SM (CTAs without a tile return before any set-up)
    k_mlp_tc<NIN><<<sms, tc::THREADS, tc::SMEM_ALLOC, s>>>(wbf16, w32, t, use_band);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc(const TableView& t, const float* w32, const uint16_t* wbf16, int n_in, int use_band,
                          cudaStream_t s) {
    if (n_in == 11) return launch_mlp_tc_t<11>(t, w32, wbf16, use_band, s);
    return launch_mlp_tc_t<2>(t, w32, wbf16, use_band, s);
}

}  // namespace pl
