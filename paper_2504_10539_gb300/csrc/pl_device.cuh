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

// Decode / encode one population.  FP16-offset stores h_i = rn(f_i - w_i rho_ref).
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::R decode(typename Traits<MODE>::S v, typename Traits<MODE>::R off) {
    if constexpr (MODE == PL_F16_OFFSET) return __half2float(v) + off;
    else return v;
}
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::S encode(typename Traits<MODE>::R v, typename Traits<MODE>::R off) {
    if constexpr (MODE == PL_F16_OFFSET) return __float2half_rn(v - off);
    else return v;
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

// Stochastic rounding of two FP32 values to FP16, packed (a -> low half, b -> high half):
// 13 dither bits are added below the FP16 mantissa's last bit and the result is truncated,
// so E[rounded] = value for values in the normal FP16 range (|v| >= 2^-14).  Bits 0-12 of
// rnd dither a, bits 16-28 dither b.
__device__ __forceinline__ __half2 sr_pack_half2(float a, float b, uint32_t rnd) {
    const float da = __uint_as_float(__float_as_uint(a) + (rnd & 0x1FFFu));
    const float db = __uint_as_float(__float_as_uint(b) + ((rnd >> 16) & 0x1FFFu));
    uint32_t r;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(db), "f"(da));
    return *reinterpret_cast<__half2*>(&r);
}
__device__ __forceinline__ __half sr_half(float a, uint32_t rnd) {
    return __float2half_rz(__uint_as_float(__float_as_uint(a) + (rnd & 0x1FFFu)));
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
    long long fix_n;        // FP16 mass restoration: signed number of rest populations shifted by one unit
    int status;          // sticky PL_ERR_* detected on the device
    int reject;          // set by the correction check pass, cleared per correction
    int applied;         // corrections applied
    int pad;
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
