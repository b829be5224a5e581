// Device-side building blocks of the lattice kernels: D2Q9 constants, the
// storage codecs, the SplitMix64 counter generator, and the deterministic
// block reduction.  Compiled only into libpinnlbm.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pinnlbm.h"

namespace pl {

// D2Q9 (arXiv 2504.10539 Sec. II-A names a lattice Boltzmann model without
// fixing it; D2Q9 is used):
//   c_0=(0,0), c_1..4=(1,0),(0,1),(-1,0),(0,-1), c_5..8=(1,1),(-1,1),(-1,-1),(1,-1)
//   w_0 = 4/9, w_1..4 = 1/9, w_5..8 = 1/36.
__host__ __device__ constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
template <typename R>
__host__ __device__ constexpr R wq(int i) {
    return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

// Storage traits: S = stored type, R = arithmetic type.
template <int MODE> struct Traits;
template <> struct Traits<PL_F64> {
    using S = double;
    using R = double;
};
template <> struct Traits<PL_F32> {
    using S = float;
    using R = float;
};
template <> struct Traits<PL_F16_OFFSET> {
    using S = __half;
    using R = float;
};

// Stored value <-> arithmetic value of FP64 / FP32 storage (the identity).  FP16-offset
// storage decodes with its reference plane (below), never through these.
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::R decode(typename Traits<MODE>::S v) {
    static_assert(MODE != PL_F16_OFFSET, "FP16-offset populations decode with their source's reference");
    return v;
}
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::S encode(typename Traits<MODE>::R v) {
    static_assert(MODE != PL_F16_OFFSET, "FP16-offset populations encode against a reference");
    return v;
}

// FP16-offset storage (a storage measure of this implementation; the paper states no number
// format).  A buffer holds ten FP16 planes: h_0..h_8 and the reference densities r.  The
// population f_i at cell x is stored relative to the reference density of the cell it
// streamed from, scaled by 2^10:
//     f_i(x) = 2^-10 h_i(x) + Wr_i r(x - c_i),
// and a step stores r(x) = fp16(rho(x)) with the populations x pushes, so each offset is the
// departure of f_i from its source cell's rest equilibrium (velocity and non-equilibrium
// terms only, a few per cent of f_i).  Wr_i = kappa w_i = (1824, 456 x4, 114 x4) / 4096 with
// kappa = 4104/4096: proportional to the lattice weights (so the offset folds into the
// equilibrium's isotropic part) and short binary fractions (so Wr_i r and kappa r are exact
// in FP32 for an FP16 r).  The scale keeps offsets down to 2^-24 in FP16's normal range, where
// a fixed 13-bit dither below the last place rounds them stochastically without bias.  A
// cell's decoded populations carry 2^-10 sum h_i + kappa r(x).
constexpr int F16_PLANES = 10;   // h_0..h_8, r
constexpr int REF_PLANE = 9;
constexpr float REF_KAPPA = 4104.0f / 4096.0f;
constexpr float F16_SCALE = 1024.0f;          // stored offset = 2^10 (f_i - Wr_i r)
constexpr float F16_UNSCALE = 1.0f / 1024.0f;
__host__ __device__ constexpr float wref(int i) {
    return i == 0 ? 1824.0f / 4096.0f : (i <= 4 ? 456.0f / 4096.0f : 114.0f / 4096.0f);
}
__host__ __device__ constexpr int planes_of(int storage) { return storage == PL_F16_OFFSET ? F16_PLANES : 9; }

// One FP16-offset cell (x, y) of a buffer f (ten planes of `plane` elements, rows of `pitch`):
// its offsets h_i (unscaled) and reference terms t_i = Wr_i r(x - c_i) (exact products), so
// that f_i = h_i + t_i and the cell's mass is A + H with A = sum t_i, H = sum h_i.  f16_refs
// gives the reference terms alone.
__device__ __forceinline__ void f16_refs(const __half* __restrict__ f, long long plane, int pitch, int nx, int ny, int x,
                                         int y, float (&t)[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const long long rm = (long long)(y == 0 ? ny - 1 : y - 1) * pitch, r0 = (long long)y * pitch,
                    rp = (long long)(y == ny - 1 ? 0 : y + 1) * pitch;
    const __half* ref = f + REF_PLANE * plane;
    t[0] = wref(0) * __half2float(ref[r0 + x]);
    t[1] = wref(1) * __half2float(ref[r0 + xm]);  // c_1 = (1, 0): from x - 1
    t[2] = wref(2) * __half2float(ref[rm + x]);   // c_2 = (0, 1): from y - 1
    t[3] = wref(3) * __half2float(ref[r0 + xp]);
    t[4] = wref(4) * __half2float(ref[rp + x]);
    t[5] = wref(5) * __half2float(ref[rm + xm]);  // c_5 = (1, 1)
    t[6] = wref(6) * __half2float(ref[rm + xp]);  // c_6 = (-1, 1)
    t[7] = wref(7) * __half2float(ref[rp + xp]);  // c_7 = (-1, -1)
    t[8] = wref(8) * __half2float(ref[rp + xm]);  // c_8 = (1, -1)
}
__device__ __forceinline__ void f16_cell(const __half* __restrict__ f, long long plane, int pitch, int nx, int ny, int x,
                                         int y, float (&h)[9], float (&t)[9]) {
    const long long o = (long long)y * pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = __half2float(f[i * plane + o]) * F16_UNSCALE;
    f16_refs(f, plane, pitch, nx, ny, x, y, t);
}
// Sums of nine terms in the walker's order.
template <typename R>
__device__ __forceinline__ R sum9(const R (&v)[9]) {
    return (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
}

__device__ __forceinline__ float psi_of(float rho, float rho0, float inv_rho0) {
    return -rho0 * expm1f(-rho * inv_rho0);
}
__device__ __forceinline__ double psi_of(double rho, double rho0, double inv_rho0) {
    return -rho0 * expm1(-rho * inv_rho0);
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) evaluated at counter k:
// the generator state after k+1 golden-gamma increments, passed through the
// published finaliser.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01_at(uint64_t seed, uint64_t k) {
    return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

// MurmurHash3's 32-bit finaliser (Appleby), used as a counter-based source of dither bits.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Stochastic rounding of two FP32 values to FP16 by the sm_100-family conversion with random
// bits (cvt.rs): a goes to the low half, b to the high half of the result.  The low half takes
// its random bits from rbits[15:0], the high half from rbits[31:16]; for an FP16 normal result
// the low 13 of those 16 bits are added below the result's last place before truncation (a
// probe of every 16-bit pattern on GB300 matched that rule exactly), and FP16 subnormal results
// round up with probability equal to the discarded fraction as well.  Uniform rbits make each
// result an unbiased rounding.
__device__ __forceinline__ uint32_t rs_pack(float a, float b, uint32_t rbits) {
    uint32_t r;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(b), "f"(a), "r"(rbits));
    return r;
}

// Per-lattice device record: reductions land here, later kernels read them,
// the host copies it out for pl_metrics.
struct DevRecord {
    // metric reduction (Eqs. 9-15)
    double mass, gmax, sum_g, sum_g2, rho_max, rho_min;
    long long count;
    // Laplace measurement
    double R_eq, rho_in, rho_out, p_in, p_out;
    // correction bookkeeping
    double mass0;        // M0
    double sum_m, sum_dr, sum_jx, sum_jy, mass_now;
    double proj, mjx, mjy;  // per-lattice constants of the apply pass (formed once, in FP64)
    int status;          // sticky PL_ERR_* detected on the device
    int reject;          // set by the correction check pass, cleared per correction
    int applied;         // corrections applied
    int band_n;          // cells in the correction's interface band (when mask_eps > 0)
};

// Deterministic block reduction of NV values per thread, fixed tree shape.
// Per-thread sum of a cell loop.  FP64 lattices sum in FP64.  FP32 terms are summed as an
// unevaluated pair hi + lo of FP32 numbers: each addition is Knuth's error-free TwoSum
// (s = hi + b exactly equals hi + b - e, e recovered with four more FP32 additions), the
// errors are collected in lo, so the pair carries about 48 significant bits.  GB300 issues
// FP64 arithmetic and FP32<->FP64 conversions at a small fraction of its FP32 rate; this keeps
// the per-cell work in FP32 and converts once per thread.  The rounding-mode intrinsics
// keep the compiler from reassociating or contracting the TwoSum.
template <typename R>
struct SumAcc;
template <>
struct SumAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double b) { v += b; }
    __device__ __forceinline__ void add_prod(double a, double b) { v += a * b; }
    __device__ __forceinline__ double value() const { return v; }
};
template <>
struct SumAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float b) {
        const float s = __fadd_rn(hi, b);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    // a b = p + q exactly (q from one FMA), both parts summed
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float q = __fmaf_rn(a, b, -p);
        add(p);
        lo = __fadd_rn(lo, q);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// op: 0 = sum, 1 = max, 2 = min.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const int (&op)[NV], double* smem /* [NV*32] */) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double w = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = op[k] == 0 ? v[k] + w : (op[k] == 1 ? fmax(v[k], w) : fmin(v[k], w));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int k = 0; k < NV; ++k) smem[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double init = op[k] == 0 ? 0.0 : (op[k] == 1 ? -INFINITY : INFINITY);
            v[k] = lane < nw ? smem[k * 32 + lane] : init;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double w = __shfl_down_sync(0xffffffffu, v[k], o);
                v[k] = op[k] == 0 ? v[k] + w : (op[k] == 1 ? fmax(v[k], w) : fmin(v[k], w));
            }
        }
    }
    __syncthreads();
}

}  // namespace pl
