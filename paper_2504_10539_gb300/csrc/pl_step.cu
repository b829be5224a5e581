// Lattice kernels of the time step (arXiv 2504.10539 Sec. II-A, Eq. 1) and
// of the initial state (Sec. III-A).
//
// Storage: structure of arrays, 9 planes of ny rows of `pitch` populations
// (x fastest, pitch = nx rounded up to 8; FP16-offset storage adds a tenth plane of
// reference densities), two buffers: a step reads the post-streaming state of buffer src
// and writes the next post-streaming state into buffer 1-src ("push").  Reads never alias
// writes, so neighbouring strips may recompute each other's densities without racing.
//
// FP16-offset storage (pl_device.cuh) keeps each population as an FP16 offset from the rest
// equilibrium of the cell it streamed from; the FP16 walker (walk_f16) decodes against those
// references, relaxes in FP32 and encodes against the relaxed cell's own new reference.
//
// Fused step kernel ("strip walker"), one pass over HBM per step:
//   - a warp owns a strip of 60 columns; lane l holds the column pair
//     (x0-2+2l, x0-1+2l), so lanes 1..30 own cells and lanes 0 and 31 carry the
//     halo; loads and stores of a pair are one aligned vector access;
//   - the warp walks its rows bottom to top, keeping the pseudopotential of three
//     rows in registers; left/right neighbours come from warp shuffles, so there
//     is no shared memory and no barrier;
//   - per cell: rho, psi, Shan-Chen force from the 3x3 psi stencil, force-shifted
//     equilibrium, BGK relaxation, and the push to the 8 neighbours; a shifted
//     plane is realigned with one shuffle so that its store is again one vector
//     access per pair.  Lanes 0 and 31 also relax their inner halo cell, whose
//     value the neighbouring owned lane pushes into its own columns;
//   - the grid is persistent: the (strip, row) pairs of the lattice are split into
//     equal contiguous ranges, one per warp, so every warp does the same work.
#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

// Launch shape of the step kernel.  Its warps are independent (no shared memory, no
// barrier).  FP16-offset: one-warp blocks, with the registers capped (96, a few bytes of
// stack) so that 21 warps fit on an SM instead of 16: that storage is bound by the latency of
// its instruction chains, and 5 more warps hide more of it (0.855 -> 0.806 ms per batched step).
// FP32/FP64: blocks of four warps, 4 (FP32) or 2 (FP64) of them per SM, the occupancy their
// register counts give anyway (FP32 is bound by HBM; one-warp blocks were slower there).
template <int MODE>
#ifndef PL_F16_MIN_BLOCKS
#define PL_F16_MIN_BLOCKS 17
#endif
struct StepCfg {
    static constexpr int threads = MODE == PL_F16_OFFSET ? 32 : 128;
    static constexpr int min_blocks = MODE == PL_F16_OFFSET ? PL_F16_MIN_BLOCKS : (MODE == PL_F32 ? 4 : 2);
};

template <int MODE> struct Pair;
template <> struct Pair<PL_F64> {
    using T = double2;
    __device__ static __forceinline__ void split(T v, double& a, double& b) { a = v.x; b = v.y; }
    __device__ static __forceinline__ T make(double a, double b) { return make_double2(a, b); }
};
template <> struct Pair<PL_F32> {
    using T = float2;
    __device__ static __forceinline__ void split(T v, float& a, float& b) { a = v.x; b = v.y; }
    __device__ static __forceinline__ T make(float a, float b) { return make_float2(a, b); }
};
template <> struct Pair<PL_F16_OFFSET> {
    using T = __half2;
    __device__ static __forceinline__ void split(T v, float& a, float& b) {
        const float2 f = __half22float2(v);
        a = f.x;
        b = f.y;
    }
    __device__ static __forceinline__ T make(float a, float b) { return __floats2half2_rn(a, b); }
};

template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::R to_r(typename Traits<MODE>::S v) {
    if constexpr (MODE == PL_F16_OFFSET) return __half2float(v);
    else return v;
}
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::S from_r(typename Traits<MODE>::R v) {
    if constexpr (MODE == PL_F16_OFFSET) return __float2half_rn(v);
    else return v;
}

// psi = rho0 (1 - exp(-rho/rho0)).  FP16 storage uses the hardware exp2; its
// cancellation error in the vapour (~1e-6 relative) is far below the storage's.
template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::R psi_step(typename Traits<MODE>::R rho, typename Traits<MODE>::R rho0,
                                                             typename Traits<MODE>::R inv_rho0) {
    if constexpr (MODE == PL_F16_OFFSET) {
        float e;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-rho * inv_rho0 * 1.4426950408889634f));
        return rho0 * (1.0f - e);
    } else {
        return psi_of(rho, rho0, inv_rho0);
    }
}

template <int MODE>
__device__ __forceinline__ typename Traits<MODE>::R recip(typename Traits<MODE>::R v) {
    if constexpr (MODE == PL_F16_OFFSET) return __fdividef(1.0f, v);
    else return typename Traits<MODE>::R(1) / v;
}

template <typename R>
struct StepK {
    R G, tau, omega, rho0, inv_rho0;
};

// One cell: populations h[9], density rho, force (fx, fy) -> o[9].
template <int MODE>
__device__ __forceinline__ void collide_cell(const typename Traits<MODE>::R (&h)[9], typename Traits<MODE>::R rho,
                                             typename Traits<MODE>::R fx, typename Traits<MODE>::R fy,
                                             const StepK<typename Traits<MODE>::R>& k,
                                             typename Traits<MODE>::R (&o)[9]) {
    using R = typename Traits<MODE>::R;
    const R jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
    const R jy = (h[2] - h[4]) + (h[5] + h[6]) - (h[7] + h[8]);
    const R inv = recip<MODE>(rho);
    const R ux = (jx + k.tau * fx) * inv;  // u + tau F / rho
    const R uy = (jy + k.tau * fy) * inv;
    const R Ap = rho * (R(1) - R(1.5) * (ux * ux + uy * uy));
    const R t3 = R(3) * rho, t45 = R(4.5) * rho;
    const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
    const R pp = ux + uy, pm = ux - uy;
    const R Sx = Ap + t45 * ux * ux, Dx = t3 * ux;
    const R Sy = Ap + t45 * uy * uy, Dy = t3 * uy;
    const R Sp = Ap + t45 * pp * pp, Dp = t3 * pp;
    const R Sm = Ap + t45 * pm * pm, Dm = t3 * pm;
    R fe[9];
    fe[0] = w0 * Ap;
    fe[1] = w1 * (Sx + Dx);
    fe[3] = w1 * (Sx - Dx);
    fe[2] = w1 * (Sy + Dy);
    fe[4] = w1 * (Sy - Dy);
    fe[5] = w2 * (Sp + Dp);
    fe[7] = w2 * (Sp - Dp);
    fe[8] = w2 * (Sm + Dm);
    fe[6] = w2 * (Sm - Dm);
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i] = h[i] + k.omega * (fe[i] - h[i]);
}

template <typename R>
struct PsiRow {
    R L, a, b, Rr;  // left neighbour, first cell, second cell, right neighbour
};

template <int MODE>
struct WalkArgs {
    const typename Traits<MODE>::S* fin;
    typename Traits<MODE>::S* fout;
    int nx, ny, pitch, nstrips, chunks;
    long long plane;
    StepK<typename Traits<MODE>::R> k;
    uint32_t seq;  // step sequence number (dither of the FP16 stochastic rounding)
};

template <int MODE>
__device__ __forceinline__ void load_row(const WalkArgs<MODE>& a, int r, int cA, int cB, bool vec,
                                         typename Pair<MODE>::T (&P)[9]) {
    using S = typename Traits<MODE>::S;
    using PT = typename Pair<MODE>::T;
    const S* row = a.fin + (long long)r * a.pitch;
    if (vec) {
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = *reinterpret_cast<const PT*>(row + i * a.plane + cA);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const S* p = row + i * a.plane;
            P[i] = Pair<MODE>::make(to_r<MODE>(p[cA]), to_r<MODE>(p[cB]));
        }
    }
}

template <int MODE>
__device__ __forceinline__ void store_pair(const WalkArgs<MODE>& a, int i, int r, int d0, bool svec, bool own0,
                                           bool own1, typename Traits<MODE>::R v0, typename Traits<MODE>::R v1) {
    using S = typename Traits<MODE>::S;
    using PT = typename Pair<MODE>::T;
    S* p = a.fout + i * a.plane + (long long)r * a.pitch + d0;
    if (svec) {
        *reinterpret_cast<PT*>(p) = Pair<MODE>::make(v0, v1);
    } else {
        if (own0) p[0] = from_r<MODE>(v0);
        if (own1) p[1] = from_r<MODE>(v1);
    }
}

// Rows [r0, r1) of strip `strip`.
template <int MODE>
__device__ void walk_segment(const WalkArgs<MODE>& a, int strip, int r0, int r1, int lane) {
    using R = typename Traits<MODE>::R;
    using PT = typename Pair<MODE>::T;
    const int nx = a.nx, ny = a.ny;
    const int ua = strip * STRIP - 2 + 2 * lane;  // unwrapped first column of this lane's pair
    const int cA = wrapi(ua, nx), cB = wrapi(ua + 1, nx);
    const bool vec = (cB == cA + 1) && ((cA & 1) == 0);
    const bool mid = lane >= 1 && lane <= 30;
    const bool own0 = mid && ua < nx, own1 = mid && ua + 1 < nx;
    const bool svec = own0 && own1 && vec;
    const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);

    PT Nx[9];
    load_row<MODE>(a, wrapi(r0 - 1, ny), cA, cB, vec, Nx);
    R hp[2][9];           // previous row (to be relaxed), decoded
    R rho_p0 = 0, rho_p1 = 0;
    PsiRow<R> A{}, B{}, C{};
    const int nrows = r1 - r0;
    for (int k = 0; k <= nrows + 1; ++k) {
        PT Cur[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Cur[i] = Nx[i];
        if (k <= nrows) {
            int rn = r0 + k;
            if (rn >= ny) rn -= ny;
            load_row<MODE>(a, rn, cA, cB, vec, Nx);  // prefetch the next row
        }
        R hc[2][9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Pair<MODE>::split(Cur[i], hc[0][i], hc[1][i]);
        // densities of the two cells
        const R rho0c = (((hc[0][0] + hc[0][1]) + (hc[0][2] + hc[0][3])) + ((hc[0][4] + hc[0][5]) + (hc[0][6] + hc[0][7])) +
                         hc[0][8]);
        const R rho1c = (((hc[1][0] + hc[1][1]) + (hc[1][2] + hc[1][3])) + ((hc[1][4] + hc[1][5]) + (hc[1][6] + hc[1][7])) +
                         hc[1][8]);
        A = B;
        B = C;
        C.a = psi_step<MODE>(rho0c, a.k.rho0, a.k.inv_rho0);
        C.b = psi_step<MODE>(rho1c, a.k.rho0, a.k.inv_rho0);
        C.L = __shfl_up_sync(0xffffffffu, C.b, 1);
        C.Rr = __shfl_down_sync(0xffffffffu, C.a, 1);
        if (k >= 2) {
            // relax row y = r0 + k - 2 with psi rows A (y-1), B (y), C (y+1)
            int y = r0 + k - 2;
            if (y >= ny) y -= ny;
            R o[2][9];
            {
                const R sx = w1 * (B.b - B.L) + w2 * ((C.b - C.L) + (A.b - A.L));
                const R sy = w1 * (C.a - A.a) + w2 * ((C.b + C.L) - (A.b + A.L));
                const R g = -a.k.G * B.a;
                collide_cell<MODE>(hp[0], rho_p0, g * sx, g * sy, a.k, o[0]);
            }
            {
                const R sx = w1 * (B.Rr - B.a) + w2 * ((C.Rr - C.a) + (A.Rr - A.a));
                const R sy = w1 * (C.b - A.b) + w2 * ((C.Rr + C.a) - (A.Rr + A.a));
                const R g = -a.k.G * B.b;
                collide_cell<MODE>(hp[1], rho_p1, g * sx, g * sy, a.k, o[1]);
            }
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            // c_x = 0 planes: own pair
            store_pair<MODE>(a, 0, y, ua, svec, own0, own1, o[0][0], o[1][0]);
            store_pair<MODE>(a, 2, yp, ua, svec, own0, own1, o[0][2], o[1][2]);
            store_pair<MODE>(a, 4, ym, ua, svec, own0, own1, o[0][4], o[1][4]);
            // c_x = +1 planes: (left lane's second cell, own first cell)
            {
                const R l1 = __shfl_up_sync(0xffffffffu, o[1][1], 1);
                const R l5 = __shfl_up_sync(0xffffffffu, o[1][5], 1);
                const R l8 = __shfl_up_sync(0xffffffffu, o[1][8], 1);
                store_pair<MODE>(a, 1, y, ua, svec, own0, own1, l1, o[0][1]);
                store_pair<MODE>(a, 5, yp, ua, svec, own0, own1, l5, o[0][5]);
                store_pair<MODE>(a, 8, ym, ua, svec, own0, own1, l8, o[0][8]);
            }
            // c_x = -1 planes: (own second cell, right lane's first cell)
            {
                const R r3 = __shfl_down_sync(0xffffffffu, o[0][3], 1);
                const R r6 = __shfl_down_sync(0xffffffffu, o[0][6], 1);
                const R r7 = __shfl_down_sync(0xffffffffu, o[0][7], 1);
                store_pair<MODE>(a, 3, y, ua, svec, own0, own1, o[1][3], r3);
                store_pair<MODE>(a, 6, yp, ua, svec, own0, own1, o[1][6], r6);
                store_pair<MODE>(a, 7, ym, ua, svec, own0, own1, o[1][7], r7);
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            hp[0][i] = hc[0][i];
            hp[1][i] = hc[1][i];
        }
        rho_p0 = rho0c;
        rho_p1 = rho1c;
    }
}

// ---------------------------------------------------------------------------------------------
// FP32-arithmetic walker (FP32 and FP16-offset storage) on packed pairs.  A lane's two cells
// are the two halves of one float2 for every population, moment and equilibrium term, and
// every addition, multiplication and FMA is one sm_100-family f32x2 instruction for both
// cells (the same IEEE rounding as the scalar FP32 operation on each half).
__device__ __forceinline__ unsigned long long f2u(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 u2f(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(d);
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

template <int MODE>
__device__ __forceinline__ float2 decode2(typename Pair<MODE>::T v) {
    if constexpr (MODE == PL_F16_OFFSET) return __half22float2(v);
    else return v;
}

template <int MODE>
__device__ __forceinline__ float2 psi2(float2 rho, const StepK<float>& k) {
    if constexpr (MODE == PL_F16_OFFSET) {
        const float2 t = rho * bc2(-k.inv_rho0 * 1.4426950408889634f);
        float ex, ey;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(t.x));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ey) : "f"(t.y));
        return fma2(bc2(-k.rho0), make_float2(ex, ey), bc2(k.rho0));
    } else {
        return make_float2(psi_of(rho.x, k.rho0, k.inv_rho0), psi_of(rho.y, k.rho0, k.inv_rho0));
    }
}

// Both cells of a pair: populations h[9], density rho, force (fx, fy) -> o[9].
// `shift` (FP16-offset storage: kappa r of the relaxed cell over omega) is subtracted from the
// equilibrium's isotropic part, so that o_i = f_i* - omega w_i shift for every i.
template <int MODE, bool SHIFT = false>
__device__ __forceinline__ void collide_pair(const float2 (&h)[9], float2 rho, float2 fx, float2 fy,
                                             const StepK<float>& k, float2 (&o)[9], float2 shift = float2{0.0f, 0.0f}) {
    const float2 jx = ((h[1] - h[3]) + (h[5] - h[6])) + (h[8] - h[7]);
    const float2 jy = ((h[2] - h[4]) + (h[5] + h[6])) - (h[7] + h[8]);
    const float2 inv = make_float2(recip<MODE>(rho.x), recip<MODE>(rho.y));
    const float2 ux = fma2(bc2(k.tau), fx, jx) * inv;  // u + tau F / rho
    const float2 uy = fma2(bc2(k.tau), fy, jy) * inv;
    const float2 usq = fma2(ux, ux, uy * uy);
    float2 Ap = rho * fma2(bc2(-1.5f), usq, bc2(1.0f));
    if constexpr (SHIFT) Ap = Ap - shift;
    // o_i = h_i + omega (f_i^eq - h_i) = (1 - omega) h_i + omega f_i^eq, with omega w_i folded
    // into the equilibrium's parts: omega f_i^eq = a_i (Ap + 4.5 rho (c_i.u)^2) +- 3 a_i rho (c_i.u),
    // a_i = omega w_i, so each population costs one add and one FMA
    const float a0 = k.omega * (4.0f / 9.0f), a1 = k.omega * (1.0f / 9.0f), a2 = k.omega * (1.0f / 36.0f);
    const float2 keep = bc2(1.0f - k.omega);
    const float2 A1 = bc2(a1) * Ap, A2 = bc2(a2) * Ap;
    const float2 q1 = bc2(4.5f * a1) * rho, q2 = bc2(4.5f * a2) * rho;
    const float2 d1 = bc2(3.0f * a1) * rho, d2 = bc2(3.0f * a2) * rho;
    const float2 pp = ux + uy, pm = ux - uy;
    const float2 Sx = fma2(q1 * ux, ux, A1), Dx = d1 * ux;
    const float2 Sy = fma2(q1 * uy, uy, A1), Dy = d1 * uy;
    const float2 Sp = fma2(q2 * pp, pp, A2), Dp = d2 * pp;
    const float2 Sm = fma2(q2 * pm, pm, A2), Dm = d2 * pm;
    o[0] = fma2(keep, h[0], bc2(a0) * Ap);
    o[1] = fma2(keep, h[1], Sx + Dx);
    o[3] = fma2(keep, h[3], Sx - Dx);
    o[2] = fma2(keep, h[2], Sy + Dy);
    o[4] = fma2(keep, h[4], Sy - Dy);
    o[5] = fma2(keep, h[5], Sp + Dp);
    o[7] = fma2(keep, h[7], Sp - Dp);
    o[8] = fma2(keep, h[8], Sm + Dm);
    o[6] = fma2(keep, h[6], Sm - Dm);
}

// Store of a lane's pair.  `split` lanes (a pair that wraps around the lattice edge, is
// not 2-element aligned, or owns one cell only) store element by element; every other lane
// owns both cells or neither, so the warp takes one branch and the vector store is
// predicated by ownership (the halo lanes 0 and 31 own nothing).
template <int MODE>
__device__ __forceinline__ void store_pair2(typename Traits<MODE>::S* p, bool split, bool own0, bool own1,
                                            typename Pair<MODE>::T v) {
    using PT = typename Pair<MODE>::T;
    if (!split) {
        if (own0) *reinterpret_cast<PT*>(p) = v;
    } else {
        if constexpr (MODE == PL_F16_OFFSET) {
            if (own0) p[0] = __low2half(v);
            if (own1) p[1] = __high2half(v);
        } else {
            if (own0) p[0] = v.x;
            if (own1) p[1] = v.y;
        }
    }
}

// Rows [r0, r1) of strip `strip`; the same walk as walk_segment.  FAST: every lane's pair
// is an aligned vector and owns both of its cells or neither (all strips but a ragged last
// one), so loads and stores need no element-wise path.
template <int MODE, bool FAST>
__device__ __forceinline__ void walk_impl2(const WalkArgs<MODE>& a, int strip, int r0, int r1, int lane) {
    using PT = typename Pair<MODE>::T;
    const int nx = a.nx, ny = a.ny;
    const int ua = strip * STRIP - 2 + 2 * lane;
    const int cA = wrapi(ua, nx), cB = wrapi(ua + 1, nx);
    const bool vec = FAST || ((cB == cA + 1) && ((cA & 1) == 0));
    const bool mid = lane >= 1 && lane <= 30;
    const bool own0 = mid && ua < nx, own1 = mid && ua + 1 < nx;
    const bool split = !FAST && !(vec && own0 == own1);
    const float w1 = 1.0f / 9.0f, w2 = 1.0f / 36.0f;
    // FAST strips index their lattice with 32-bit element offsets (the caller checks that 9
    // planes fit): each access is one multiply-add of the plane offset plus one widening
    // address computation, instead of 64-bit arithmetic per access.
    using S = typename Traits<MODE>::S;
    const uint32_t planeU = (uint32_t)a.plane, pitchU = (uint32_t)a.pitch;
    auto load_fast = [&](int r, PT (&P)[9]) {
        const uint32_t off = (uint32_t)r * pitchU + (uint32_t)cA;
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = *reinterpret_cast<const PT*>(a.fin + (off + (uint32_t)i * planeU));
    };

    PT Nx[9];
    if constexpr (FAST) load_fast(wrapi(r0 - 1, ny), Nx);
    else load_row<MODE>(a, wrapi(r0 - 1, ny), cA, cB, vec, Nx);
    float2 hp[9];  // previous row (to be relaxed), decoded
    float2 rho_p = make_float2(0.0f, 0.0f), sh_p = make_float2(0.0f, 0.0f);
    PsiRow<float> A{}, B{}, C{};
    const int nrows = r1 - r0;
    for (int k = 0; k <= nrows + 1; ++k) {
        PT Cur[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Cur[i] = Nx[i];
        if (k <= nrows) {
            int rn = r0 + k;
            if (rn >= ny) rn -= ny;
            if constexpr (FAST) load_fast(rn, Nx);  // prefetch the next row
            else load_row<MODE>(a, rn, cA, cB, vec, Nx);
        }
        float2 hc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) hc[i] = decode2<MODE>(Cur[i]);
        const float2 shc = (((hc[0] + hc[1]) + (hc[2] + hc[3])) + ((hc[4] + hc[5]) + (hc[6] + hc[7]))) + hc[8];
        const float2 rhoc = shc;
        A = B;
        B = C;
        const float2 ps = psi2<MODE>(rhoc, a.k);
        C.a = ps.x;
        C.b = ps.y;
        C.L = __shfl_up_sync(0xffffffffu, C.b, 1);
        C.Rr = __shfl_down_sync(0xffffffffu, C.a, 1);
        if (k >= 2) {
            int y = r0 + k - 2;
            if (y >= ny) y -= ny;
            // Shan-Chen force of both cells from the 3x3 psi stencil (rows A = y-1, B = y, C = y+1)
            const float sx0 = w1 * (B.b - B.L) + w2 * ((C.b - C.L) + (A.b - A.L));
            const float sy0 = w1 * (C.a - A.a) + w2 * ((C.b + C.L) - (A.b + A.L));
            const float sx1 = w1 * (B.Rr - B.a) + w2 * ((C.Rr - C.a) + (A.Rr - A.a));
            const float sy1 = w1 * (C.b - A.b) + w2 * ((C.Rr + C.a) - (A.Rr + A.a));
            const float g0 = -a.k.G * B.a, g1 = -a.k.G * B.b;
            float2 o[9];
            collide_pair<MODE>(hp, rho_p, make_float2(g0 * sx0, g1 * sx1), make_float2(g0 * sy0, g1 * sy1), a.k, o);
            // BGK conserves mass; take the rest population from that balance so the FP32
            // weights (which do not sum to one exactly) leave no systematic drift.
            o[0] = sh_p - (((o[1] + o[2]) + (o[3] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
            PT out[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i] = o[i];
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            auto dst = [&](int i, int row) -> S* {
                if constexpr (FAST) return a.fout + ((uint32_t)row * pitchU + (uint32_t)ua + (uint32_t)i * planeU);
                else return a.fout + i * a.plane + (long long)row * a.pitch + ua;
            };
            // c_x = 0 planes: own pair
            store_pair2<MODE>(dst(0, y), split, own0, own1, out[0]);
            store_pair2<MODE>(dst(2, yp), split, own0, own1, out[2]);
            store_pair2<MODE>(dst(4, ym), split, own0, own1, out[4]);
            // c_x = +1 planes: (left lane's second cell, own first cell);
            // c_x = -1 planes: (own second cell, right lane's first cell)
            {
                const float l1 = __shfl_up_sync(0xffffffffu, o[1].y, 1);
                const float l5 = __shfl_up_sync(0xffffffffu, o[5].y, 1);
                const float l8 = __shfl_up_sync(0xffffffffu, o[8].y, 1);
                const float r3 = __shfl_down_sync(0xffffffffu, o[3].x, 1);
                const float r6 = __shfl_down_sync(0xffffffffu, o[6].x, 1);
                const float r7 = __shfl_down_sync(0xffffffffu, o[7].x, 1);
                store_pair2<MODE>(dst(1, y), split, own0, own1, make_float2(l1, o[1].x));
                store_pair2<MODE>(dst(5, yp), split, own0, own1, make_float2(l5, o[5].x));
                store_pair2<MODE>(dst(8, ym), split, own0, own1, make_float2(l8, o[8].x));
                store_pair2<MODE>(dst(3, y), split, own0, own1, make_float2(o[3].y, r3));
                store_pair2<MODE>(dst(6, yp), split, own0, own1, make_float2(o[6].y, r6));
                store_pair2<MODE>(dst(7, ym), split, own0, own1, make_float2(o[7].y, r7));
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) hp[i] = hc[i];
        rho_p = rhoc;
        sh_p = shc;
    }
}

// ---------------------------------------------------------------------------------------------
// FP16-offset walker: the strip walk of walk_impl2 on packed FP32 pairs, with the storage of
// pl_device.cuh.  A population arriving at cell x is decoded against the reference density of
// the cell it streamed from, f_i = 2^-10 h_i + Wr_i r(x - c_i); the relaxed pair stores its new
// reference r(x) = fp16(rho(x)) in plane 9 and pushes h_i = 2^10 (f_i* - Wr_i r(x)).  The reference
// rows y-1, y, y+1 are held as packed FP16 pairs: the lane's own pair and, in a second word,
// its left and right neighbours (the adjacent lanes' values by shuffle; lanes 0 and 31 read
// their one outer column from memory), loaded one row ahead of the populations.
//
// Mass: the relaxed cell's populations carry 2^-10 sum h_i + kappa r(x) once decoded (kappa r
// exact in FP32), so the rest offset takes 2^10 (rho - kappa r(x)) - sum_{i>0} h_i: the cell's
// mass to within FP32 rounding of its density sum and one zero-mean rounding of the rest
// offset.  Every offset is rounded stochastically, so rounding biases neither the mass nor the
// momentum a population carries.
__device__ __forceinline__ uint32_t h2u(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ __half2 u2h(uint32_t v) { return *reinterpret_cast<__half2*>(&v); }

// A reference row in FP32: the lane's own pair M = (r(a), r(b)) and its outer neighbours
// L = r(a - 1), R = r(b + 1).
struct RefRow {
    float2 M;
    float L, R;
};

template <bool FAST>
__device__ __forceinline__ void walk_f16(const WalkArgs<PL_F16_OFFSET>& a, int strip, int r0, int r1, int lane) {
    const int nx = a.nx, ny = a.ny;
    const int ua = strip * STRIP - 2 + 2 * lane;
    const int cA = wrapi(ua, nx), cB = wrapi(ua + 1, nx);
    const bool vec = FAST || ((cB == cA + 1) && ((cA & 1) == 0));
    const bool mid = lane >= 1 && lane <= 30;
    const bool own0 = mid && ua < nx, own1 = mid && ua + 1 < nx;
    const bool split = !FAST && !(vec && own0 == own1);
    const bool halo = lane == 0 || lane == 31;
    const int cX = lane == 0 ? wrapi(ua - 1, nx) : wrapi(ua + 2, nx);  // a halo lane's outer column
    const float w1 = 1.0f / 9.0f, w2 = 1.0f / 36.0f;
    // the walk runs in units of 2^-10 (populations F = 2^10 f, densities rho_s = 2^10 rho):
    // a stored offset h is then F - 2^10 Wr_i r directly
    const float W0 = F16_SCALE * wref(0), W1 = F16_SCALE * wref(1), W2 = F16_SCALE * wref(5);
    const uint32_t planeU = (uint32_t)a.plane, pitchU = (uint32_t)a.pitch;
    // element offset of column 0 of row r of plane i (FAST strips: 32 bits, checked by the caller)
    auto row_off = [&](int i, int r) -> long long {
        if constexpr (FAST) return (long long)((uint32_t)r * pitchU + (uint32_t)i * planeU);
        else return (long long)i * a.plane + (long long)r * a.pitch;
    };
    auto ld_pair = [&](const __half* row) -> uint32_t {
        if (vec) return *reinterpret_cast<const uint32_t*>(row + cA);
        return (uint32_t)__half_as_ushort(row[cA]) | ((uint32_t)__half_as_ushort(row[cB]) << 16);
    };
    auto load_pops = [&](int r, uint32_t (&P)[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) P[i] = ld_pair(a.fin + row_off(i, r));
    };
    auto load_ref = [&](int r, uint32_t& own, uint32_t& ext) {
        const __half* row = a.fin + row_off(REF_PLANE, r);
        own = ld_pair(row);
        ext = halo ? (uint32_t)__half_as_ushort(row[cX]) : 0u;
    };
    auto ref_row = [&](uint32_t own, uint32_t ext) -> RefRow {
        const uint32_t up = __shfl_up_sync(0xffffffffu, own, 1);    // left lane's pair
        const uint32_t dn = __shfl_down_sync(0xffffffffu, own, 1);  // right lane's pair
        uint32_t sd = __byte_perm(up, dn, 0x5432);                  // (its b, right lane's a)
        if (lane == 0) sd = (sd & 0xFFFF0000u) | ext;
        if (lane == 31) sd = (sd & 0x0000FFFFu) | (ext << 16);
        const float2 s2 = __half22float2(u2h(sd));
        return RefRow{__half22float2(u2h(own)), s2.x, s2.y};
    };
    auto store = [&](__half* p, uint32_t v) {
        if (!split) {
            if (own0) *reinterpret_cast<uint32_t*>(p) = v;
        } else {
            if (own0) p[0] = __ushort_as_half((unsigned short)(v & 0xFFFFu));
            if (own1) p[1] = __ushort_as_half((unsigned short)(v >> 16));
        }
    };

    // populations of row r0-1 (decoded first), references of rows r0-2, r0-1, r0 (its
    // neighbourhood) and r0+1 (pending)
    uint32_t Nx[9];
    load_pops(wrapi(r0 - 1, ny), Nx);
    RefRow rm, rc, rp;
    uint32_t pend_own, pend_ext;
    {
        uint32_t o, e;
        load_ref(wrapi(r0 - 2, ny), o, e);
        rm = ref_row(o, e);
        load_ref(wrapi(r0 - 1, ny), o, e);
        rc = ref_row(o, e);
        load_ref(wrapi(r0, ny), o, e);
        rp = ref_row(o, e);
        load_ref(wrapi(r0 + 1, ny), pend_own, pend_ext);
    }
    float2 fp[9];  // previous row (to be relaxed), decoded
    float2 rho_p = make_float2(0.0f, 0.0f);
    // pseudopotential of rows y-1, y, y+1 (the pair's own cells; the neighbours come by
    // shuffle when the force is formed, so that fewer values stay live across rows)
    float2 PA = make_float2(0.0f, 0.0f), PB = PA, PC = PA;
    const int nrows = r1 - r0;
    for (int k = 0; k <= nrows + 1; ++k) {
        uint32_t Cur[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Cur[i] = Nx[i];
        if (k <= nrows) {
            int rn = r0 + k;
            if (rn >= ny) rn -= ny;
            load_pops(rn, Nx);                       // prefetch the next row
        }
        // decode row r0+k-1 against the references of rows r0+k-2 (rm), r0+k-1 (rc), r0+k (rp):
        // F_i = h_i + 2^10 Wr_i r(x - c_i), one FMA each (the shifted views per half)
        float2 fc[9];
        {
            float2 h[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = __half22float2(u2h(Cur[i]));
            fc[0] = fma2(bc2(W0), rc.M, h[0]);
            fc[1] = make_float2(fmaf(W1, rc.L, h[1].x), fmaf(W1, rc.M.x, h[1].y));   // c_1 = (1, 0): from x - 1
            fc[3] = make_float2(fmaf(W1, rc.M.y, h[3].x), fmaf(W1, rc.R, h[3].y));
            fc[2] = fma2(bc2(W1), rm.M, h[2]);                                        // c_y = +1: from row y - 1
            fc[5] = make_float2(fmaf(W2, rm.L, h[5].x), fmaf(W2, rm.M.x, h[5].y));
            fc[6] = make_float2(fmaf(W2, rm.M.y, h[6].x), fmaf(W2, rm.R, h[6].y));
            fc[4] = fma2(bc2(W1), rp.M, h[4]);                                        // c_y = -1: from row y + 1
            fc[8] = make_float2(fmaf(W2, rp.L, h[8].x), fmaf(W2, rp.M.x, h[8].y));
            fc[7] = make_float2(fmaf(W2, rp.M.y, h[7].x), fmaf(W2, rp.R, h[7].y));
        }
        // slide the reference window: the pending row is complete now
        rm = rc;
        rc = rp;
        rp = ref_row(pend_own, pend_ext);
        if (k < nrows) load_ref(wrapi(r0 + k + 2, ny), pend_own, pend_ext);  // decoded two iterations on
        const float2 rhoc = (((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + (fc[6] + fc[7]))) + fc[8];
        PA = PB;
        PB = PC;
        PC = psi2<PL_F16_OFFSET>(rhoc * bc2(F16_UNSCALE), a.k);
        if (k >= 2) {
            int y = r0 + k - 2;
            if (y >= ny) y -= ny;
            PsiRow<float> A, B, C;
            A.a = PA.x, A.b = PA.y, B.a = PB.x, B.b = PB.y, C.a = PC.x, C.b = PC.y;
            A.L = __shfl_up_sync(0xffffffffu, A.b, 1);
            A.Rr = __shfl_down_sync(0xffffffffu, A.a, 1);
            B.L = __shfl_up_sync(0xffffffffu, B.b, 1);
            B.Rr = __shfl_down_sync(0xffffffffu, B.a, 1);
            C.L = __shfl_up_sync(0xffffffffu, C.b, 1);
            C.Rr = __shfl_down_sync(0xffffffffu, C.a, 1);
            const float sx0 = w1 * (B.b - B.L) + w2 * ((C.b - C.L) + (A.b - A.L));
            const float sy0 = w1 * (C.a - A.a) + w2 * ((C.b + C.L) - (A.b + A.L));
            const float sx1 = w1 * (B.Rr - B.a) + w2 * ((C.Rr - C.a) + (A.Rr - A.a));
            const float sy1 = w1 * (C.b - A.b) + w2 * ((C.Rr + C.a) - (A.Rr + A.a));
            // the force in the walk's units (the collision takes tau F / rho with rho scaled)
            const float g0 = -a.k.G * F16_SCALE * B.a, g1 = -a.k.G * F16_SCALE * B.b;
            // the pair's new reference; the relaxation then gives the stored offsets directly
            // (o_i = F_i* - 2^10 Wr_i r, the shift 2^10 kappa r / omega taken off the isotropic part)
            uint32_t rq;
            {
                const float2 rho = rho_p * bc2(F16_UNSCALE);
                asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(rq) : "f"(rho.y), "f"(rho.x));
            }
            const float2 rqf = __half22float2(u2h(rq));
            float2 o[9];
            collide_pair<PL_F16_OFFSET, true>(fp, rho_p, make_float2(g0 * sx0, g1 * sx1), make_float2(g0 * sy0, g1 * sy1),
                                              a.k, o, bc2(REF_KAPPA * F16_SCALE * a.k.tau) * rqf);
            // every offset rounded stochastically (unbiased: no drift of mass or momentum from
            // rounding) by the conversion with random bits, one 32-bit word per pair and
            // population: a counter-based hash of the pair's position and the lattice's step
            // count, stepped by a linear congruential sequence per population
            const uint32_t rnd =
                fmix32(((uint32_t)ua * 0x85EBCA77u) ^ ((uint32_t)y * 0xC2B2AE3Du) ^ (a.seq * 0x27D4EB2Fu));
            uint32_t st = rnd;
            uint32_t out[9];
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                st = st * 1664525u + 1013904223u;
                out[i] = rs_pack(o[i].x, o[i].y, st);
                unsigned short lo, hi;
                asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(out[i]));
                asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(s0) : "h"(lo));
                asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(s1) : "h"(hi));
            }
            // rest offset: the cell's mass minus what the pushed populations carry
            const float2 rest = (rho_p - bc2(REF_KAPPA * F16_SCALE) * rqf) - make_float2(s0, s1);
            out[0] = rs_pack(rest.x, rest.y, rnd);
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            auto dst = [&](int i, int row) -> __half* { return a.fout + row_off(i, row) + ua; };
            // c_x = 0 planes and the reference: own pair
            store(dst(0, y), out[0]);
            store(dst(REF_PLANE, y), rq);
            store(dst(2, yp), out[2]);
            store(dst(4, ym), out[4]);
            // c_x = +1 planes: (high half of the left lane's pair, low half of ours);
            // c_x = -1 planes: (high half of ours, low half of the right lane's pair)
            const uint32_t u1 = __shfl_up_sync(0xffffffffu, out[1], 1);
            const uint32_t u5 = __shfl_up_sync(0xffffffffu, out[5], 1);
            const uint32_t u8 = __shfl_up_sync(0xffffffffu, out[8], 1);
            const uint32_t d3 = __shfl_down_sync(0xffffffffu, out[3], 1);
            const uint32_t d6 = __shfl_down_sync(0xffffffffu, out[6], 1);
            const uint32_t d7 = __shfl_down_sync(0xffffffffu, out[7], 1);
            store(dst(1, y), __byte_perm(u1, out[1], 0x5432));
            store(dst(5, yp), __byte_perm(u5, out[5], 0x5432));
            store(dst(8, ym), __byte_perm(u8, out[8], 0x5432));
            store(dst(3, y), __byte_perm(out[3], d3, 0x5432));
            store(dst(6, yp), __byte_perm(out[6], d6, 0x5432));
            store(dst(7, ym), __byte_perm(out[7], d7, 0x5432));
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) fp[i] = fc[i];
        rho_p = rhoc;
    }
}

// Whether strip `strip` of a lattice takes the FP16 vector path: every pair of the strip is an
// aligned vector that owns both of its cells or neither (lanes past the lattice's last column
// read wrapped columns, needed only for the psi of their neighbours, and store nothing) and
// ten planes fit 32-bit element offsets.  True for every strip of a lattice with even nx (and
// planes below 2^32 / 10 elements); warp-uniform.
__device__ __forceinline__ bool f16_fast_strip(int nx, long long plane, int strip, int lane) {
    const int ua = strip * STRIP - 2 + 2 * lane;
    const int cA = wrapi(ua, nx), cB = wrapi(ua + 1, nx);
    const bool mid = lane >= 1 && lane <= 30;
    const bool own0 = mid && ua < nx, own1 = mid && ua + 1 < nx;
    const bool fast = (cB == cA + 1) && ((cA & 1) == 0) && own0 == own1 && (long long)F16_PLANES * plane <= 0xFFFFFFFFll;
    return __all_sync(0xffffffffu, fast);
}

template <int MODE>
__device__ void walk_segment2(const WalkArgs<MODE>& a, int strip, int r0, int r1, int lane) {
    // (FP32 storage is bound by HBM, not by issue: it keeps one copy of the walk and its
    // register count, and with it four blocks per SM)
    if constexpr (MODE == PL_F16_OFFSET) {
        // the vector path only: the other strips are k_step_edge's
        if (f16_fast_strip(a.nx, a.plane, strip, lane)) walk_f16<true>(a, strip, r0, r1, lane);
    } else {
        walk_impl2<MODE, false>(a, strip, r0, r1, lane);
    }
}

// Persistent table kernel: physical warp w processes virtual warps w, w+P, w+2P, ...
// Virtual warp v belongs to the lattice j with warp_pre[j] <= v < warp_pre[j+1]; its
// local index l walks strip (l mod nstrips) over row chunk (l / nstrips).  The rows of a
// lattice are cut into equal chunks, the same cut in every strip, so the warps of one
// chunk (consecutive virtual warps) start together and advance one row per iteration:
// horizontally adjacent strips touch the sectors they share (halo columns, partial
// sectors at strip edges) at the same time and those are served from L2, and each row
// of a plane is read as one contiguous sweep.
__device__ __forceinline__ int find_seg(const long long* __restrict__ pre, int n, long long v) {
    int lo = 0, hi = n;  // pre[lo] <= v < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int MODE>
__global__ void __launch_bounds__(StepCfg<MODE>::threads, StepCfg<MODE>::min_blocks) k_step(TableView t, int parity) {
    using S = typename Traits<MODE>::S;
    using R = typename Traits<MODE>::R;
    const int lane = threadIdx.x & 31;
    constexpr int TH = StepCfg<MODE>::threads;
    const long long P = (long long)gridDim.x * (TH / 32);
    const long long total = t.hdr->total_warps;
    const int n = t.hdr->n;
    const uint32_t seq = t.seq[parity];
    if (blockIdx.x == 0 && threadIdx.x == 0) t.seq[parity ^ 1] = seq + 1u;
    // when the table has fewer virtual warps than the grid has warps, consecutive virtual warps
    // go to different blocks (SMs), so a small lattice's few warps spread over as many SMs as
    // they can instead of filling the first blocks; else the warps of a block take
    // consecutive virtual warps (neighbouring strips, whose shared columns then hit in L1)
    const long long w = threadIdx.x >> 5;
    const long long vw0 = total < P ? w * gridDim.x + blockIdx.x : (long long)blockIdx.x * (TH / 32) + w;
    for (long long vw = vw0; vw < total; vw += P) {
        const int j = find_seg(t.warp_pre, n, vw);
        const LatDesc& d = t.d[j];
        const long long local = vw - t.warp_pre[j];
        const int strip = (int)(local % d.nstrips);
        const long long chunk = local / d.nstrips;
        const int r0 = (int)(chunk * d.ny / d.chunks);
        const int r1 = (int)((chunk + 1) * d.ny / d.chunks);
        if (r1 <= r0) continue;
        WalkArgs<MODE> a;
        const int src = d.phase ^ parity;
        a.fin = static_cast<const S*>(d.pops[src]);
        a.fout = static_cast<S*>(d.pops[1 - src]);
        a.nx = d.nx;
        a.ny = d.ny;
        a.pitch = d.pitch;
        a.nstrips = d.nstrips;
        a.chunks = d.chunks;
        a.plane = d.plane;
        a.k = StepK<R>{R(d.G), R(d.tau), R(1.0 / d.tau), R(d.rho0), R(1.0 / d.rho0)};
        a.seq = seq - d.seq0;  // the lattice's own step count: the same alone or in a batch
        if constexpr (MODE == PL_F64) walk_segment<MODE>(a, strip, r0, r1, lane);
        else walk_segment2<MODE>(a, strip, r0, r1, lane);
    }
}

// FP16-offset strips off the vector path (ragged or wrapping pairs of odd-nx lattices, planes
// beyond 32-bit offsets), element by element.  A kernel of its own, so that its register needs
// do not spill the vector path's; it walks only the lattices the header counts and returns at
// once when there are none.
__global__ void __launch_bounds__(128) k_step_edge(TableView t, int parity) {
    if (t.hdr->edge_lattices == 0) return;
    const int lane = threadIdx.x & 31;
    const long long P = (long long)gridDim.x * (blockDim.x / 32);
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n = t.hdr->n;
    const uint32_t seq = t.seq[parity];
    for (int j = 0; j < n; ++j) {
        const LatDesc& d = t.d[j];
        if (!f16_edge_lattice(d.nx, d.plane)) continue;
        const long long nvw = (long long)d.nstrips * d.chunks;
        for (long long local = w0; local < nvw; local += P) {
            const int strip = (int)(local % d.nstrips);
            const long long chunk = local / d.nstrips;
            const int r0 = (int)(chunk * d.ny / d.chunks);
            const int r1 = (int)((chunk + 1) * d.ny / d.chunks);
            if (r1 <= r0 || f16_fast_strip(d.nx, d.plane, strip, lane)) continue;
            WalkArgs<PL_F16_OFFSET> a;
            const int src = d.phase ^ parity;
            a.fin = static_cast<const __half*>(d.pops[src]);
            a.fout = static_cast<__half*>(d.pops[1 - src]);
            a.nx = d.nx;
            a.ny = d.ny;
            a.pitch = d.pitch;
            a.nstrips = d.nstrips;
            a.chunks = d.chunks;
            a.plane = d.plane;
            a.k = StepK<float>{float(d.G), float(d.tau), float(1.0 / d.tau), float(d.rho0), float(1.0 / d.rho0)};
            a.seq = seq - d.seq0;
            walk_f16<false>(a, strip, r0, r1, lane);
        }
    }
}

template <int MODE>
static int capacity_t() {
    static int cap = 0;
    if (!cap) {
        int dev = 0, sms = 0, bps = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_step<MODE>, StepCfg<MODE>::threads, 0) != cudaSuccess ||
            bps < 1)
            bps = 1;
        cap = bps * sms * (StepCfg<MODE>::threads / 32);
    }
    return cap;
}

int step_capacity_warps(int storage) {
    switch (storage) {
        case PL_F64: return capacity_t<PL_F64>();
        case PL_F32: return capacity_t<PL_F32>();
        default: return capacity_t<PL_F16_OFFSET>();
    }
}

template <int MODE>
static cudaError_t launch_step_t(const TableView& t, int parity, cudaStream_t s) {
    const int blocks = capacity_t<MODE>() / (StepCfg<MODE>::threads / 32);
    k_step<MODE><<<blocks, StepCfg<MODE>::threads, 0, s>>>(t, parity);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_step_tab(const TableView& t, int storage, int parity, cudaStream_t s, bool edge) {
    switch (storage) {
        case PL_F64: return launch_step_t<PL_F64>(t, parity, s);
        case PL_F32: return launch_step_t<PL_F32>(t, parity, s);
        case PL_F16_OFFSET: {
            cudaError_t e = launch_step_t<PL_F16_OFFSET>(t, parity, s);
            if (e != cudaSuccess || !edge) return e;
            static int sms = 0;
            if (!sms) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (sms < 1) sms = 1;
            }
            k_step_edge<<<sms, 128, 0, s>>>(t, parity);
            note_launches(1);
            return cudaGetLastError();
        }
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Initial state (Sec. III-A): tanh droplet profile(s), counter-based noise, f_i = w_i rho.

__device__ __forceinline__ double min_image(double d, double n) {
    double a = fabs(fmod(d, n));
    return a > 0.5 * n ? n - a : a;
}

// Density of the initial droplet state, rho[y*nx + x] in FP64.
__global__ void k_droplet_rho(int nx, int ny, const pl_droplet* __restrict__ d, int n, double rho_in, double rho_out,
                              double width, double noise_amp, uint64_t seed, double* __restrict__ rho) {
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
        rho[c] = rho_out + (rho_in - rho_out) * best + noise_amp * (2.0 * uniform01_at(seed, (uint64_t)c) - 1.0);
    }
}

// Fluid at rest, f_i = w_i rho (FP64 / FP32 storage).
template <int MODE>
__global__ void k_init_from_rho(typename Traits<MODE>::S* __restrict__ f, int nx, int ny, int pitch, long long plane,
                                const double* __restrict__ rho) {
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long o = (c / nx) * pitch + c % nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * plane + o] = encode<MODE>(R(wq<double>(i) * rho[c]));
    }
}

// FP16-offset storage: reference plane r = fp16(rho) of a density field given in FP64.
__global__ void k_ref_from_rho(__half* __restrict__ ref, int nx, int ny, int pitch, const double* __restrict__ rho) {
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        ref[(c / nx) * pitch + c % nx] = __double2half(rho[c]);
}

// Reference term Wr_i r(x - c_i) of population i at cell (x, y), exact in FP64.
__device__ __forceinline__ double ref_term(const __half* __restrict__ ref, int nx, int ny, int pitch, int x, int y, int i) {
    const int xs = wrapi(x - cx(i), nx), ys = wrapi(y - cy(i), ny);
    return (double)wref(i) * (double)__half2float(ref[(long long)ys * pitch + xs]);
}

// FP16-offset storage of a fluid at rest, f_i = w_i rho, against the reference plane: each
// moving population rounded to nearest, the rest population taking the cell's density minus
// what the others carry (so the stored mass of a cell is rho within one rounding of h_0).
__global__ void k_f16_encode_rest(__half* __restrict__ f, int nx, int ny, int pitch, long long plane,
                                  const double* __restrict__ rho) {
    const __half* ref = f + REF_PLANE * plane;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const long long o = (long long)y * pitch + x;
        double carried = ref_term(ref, nx, ny, pitch, x, y, 0);
        for (int i = 1; i < 9; ++i) {
            const double t = ref_term(ref, nx, ny, pitch, x, y, i);
            const __half h = __double2half((wq<double>(i) * rho[c] - t) * (double)F16_SCALE);
            f[i * plane + o] = h;
            carried += (double)__half2float(h) * (double)F16_UNSCALE + t;
        }
        f[o] = __double2half((rho[c] - carried) * (double)F16_SCALE);
    }
}

// FP64 dense exchange array <-> one pitched storage plane (plane index `i`).  FP16-offset
// storage decodes f_i = 2^-10 h_i + Wr_i r(x - c_i) and encodes h_i = fp16(2^10 (f_i - Wr_i
// r(x - c_i))) (to nearest, in FP64) against the reference plane, which k_ref_from_rho has set
// first.
template <int MODE>
__global__ void k_plane_convert(typename Traits<MODE>::S* __restrict__ f, int nx, int ny, int pitch, long long plane,
                                int i, double* __restrict__ buf, int to_f64) {
    using R = typename Traits<MODE>::R;
    const long long N = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const long long o = i * plane + (long long)y * pitch + x;
        if constexpr (MODE == PL_F16_OFFSET) {
            const double t = ref_term(f + REF_PLANE * plane, nx, ny, pitch, x, y, i);
            if (to_f64) buf[c] = (double)__half2float(f[o]) * (double)F16_UNSCALE + t;
            else f[o] = __double2half((buf[c] - t) * (double)F16_SCALE);
        } else {
            if (to_f64) buf[c] = (double)decode<MODE>(f[o]);
            else f[o] = encode<MODE>(R(buf[c]));
        }
    }
}

// acc = buf (first) or acc + buf: the density of a state uploaded one plane at a time.
__global__ void k_accumulate(double* __restrict__ acc, const double* __restrict__ buf, long long N, int first) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        acc[c] = first ? buf[c] : acc[c] + buf[c];
}

static int grid_for(long long N) {
    long long b = (N + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

cudaError_t launch_init_from_rho(const LatticeView& v, const PhysParams& p, int cur, const double* d_rho,
                                 cudaStream_t s) {
    (void)p;
    const int g = grid_for((long long)v.nx * v.ny);
    switch (v.storage) {
        case PL_F64:
            k_init_from_rho<PL_F64><<<g, 256, 0, s>>>(static_cast<double*>(v.pops[cur]), v.nx, v.ny, v.pitch, v.plane, d_rho);
            note_launches(1);
            break;
        case PL_F32:
            k_init_from_rho<PL_F32><<<g, 256, 0, s>>>(static_cast<float*>(v.pops[cur]), v.nx, v.ny, v.pitch, v.plane, d_rho);
            note_launches(1);
            break;
        case PL_F16_OFFSET: {
            __half* f = static_cast<__half*>(v.pops[cur]);
            k_ref_from_rho<<<g, 256, 0, s>>>(f + REF_PLANE * v.plane, v.nx, v.ny, v.pitch, d_rho);
            k_f16_encode_rest<<<g, 256, 0, s>>>(f, v.nx, v.ny, v.pitch, v.plane, d_rho);
            note_launches(2);
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The droplet density goes through the lattice's scratch (>= 8 N bytes) as FP64.
cudaError_t launch_init_droplets(const LatticeView& v, const PhysParams& p, int cur, int n, double rho_in,
                                 double rho_out, double width, double noise_amp, uint64_t seed, cudaStream_t s) {
    double* rho = static_cast<double*>(v.rho);
    k_droplet_rho<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v.nx, v.ny, v.droplets, n, rho_in, rho_out, width,
                                                                   noise_amp, seed, rho);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_init_from_rho(v, p, cur, rho, s);
}

template <int MODE>
static void convert_t(const LatticeView& v, int cur, double* d_buf, int i, int to_f64, cudaStream_t s) {
    using S = typename Traits<MODE>::S;
    k_plane_convert<MODE><<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(static_cast<S*>(v.pops[cur]), v.nx, v.ny,
                                                                           v.pitch, v.plane, i, d_buf, to_f64);
}

cudaError_t launch_state_convert(const LatticeView& v, const PhysParams& p, int cur, double* d_buf, int i, int to_f64,
                                 cudaStream_t s) {
    (void)p;
    switch (v.storage) {
        case PL_F64: convert_t<PL_F64>(v, cur, d_buf, i, to_f64, s); break;
        case PL_F32: convert_t<PL_F32>(v, cur, d_buf, i, to_f64, s); break;
        case PL_F16_OFFSET: convert_t<PL_F16_OFFSET>(v, cur, d_buf, i, to_f64, s); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_state_accumulate(const LatticeView& v, double* d_acc, const double* d_buf, int first,
                                    cudaStream_t s) {
    const long long N = (long long)v.nx * v.ny;
    k_accumulate<<<grid_for(N), 256, 0, s>>>(d_acc, d_buf, N, first);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_state_ref(const LatticeView& v, int cur, const double* d_rho, cudaStream_t s) {
    if (v.storage != PL_F16_OFFSET) return cudaSuccess;
    __half* f = static_cast<__half*>(v.pops[cur]);
    k_ref_from_rho<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(f + REF_PLANE * v.plane, v.nx, v.ny, v.pitch, d_rho);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pl
