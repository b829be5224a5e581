// Training of the correction network on the lattice state, arXiv 2504.10539 Sec. II-C step 2
// with the composite loss of Eqs. 3-8 and the hyper-parameters of Sec. III-B, on CUDA cores:
// FP32 for FP32 / FP16-offset lattices, FP64 for FP64 lattices.
//
// What one epoch computes (the readings of the paper's open points are fixed here):
//   samples  every cell, input (x^, y^) = the cell centre mapped to [-1, 1]; one epoch is one
//            gradient step on the loss over all cells;
//   targets  rho = sum f_i, u = j / rho of the state when training starts;
//   L_data   (Eq. 4) mean over the cells of |N - (rho, u_x, u_y)|^2;
//   L_phys   (Eqs. 5-7) mean of r_c^2 + |r_m|^2 with r_c = div(rho u), r_m = div(rho u u) +
//            grad p, on the network's own fields and their spatial derivatives; no time
//            derivative (N has no time input), p = rho/3 + G psi^2/6, stress taken as zero;
//   L_int    (Eq. 8) mean over the interface cells (lattice |grad rho| above the Eq. 9
//            threshold) of -alpha1 q + alpha2 q^2, q = |grad rho_N|^2: the signs the text
//            describes (Eq. 8 as printed is unbounded below);
//   d/dx     in lattice units, (2 / nx) d/dx^;
//   update   Adam (lr 3e-4 in Sec. III-B), moments kept across calls.
//
// The spatial derivatives of the network are forward tangents: every layer carries three
// rows per sample, its value and its derivatives along x^ and y^ (z_d = W a_d, a_d =
// tanh'(z) z_d).  The reverse pass runs through all three rows; the only coupling between
// them is tanh's second derivative:  dL/dz = s dL/da - 2 a sum_d a_d dL/da_d, s = 1 - a^2.
//
// Kernel layout.  A CTA of 256 threads (one per SM) takes tiles of T samples (T = 16 in FP32,
// 8 in FP64), i.e. 3T rows, and keeps every hidden layer's rows of the tile in shared memory
// for the reverse pass.  The dense layers are register-tiled loops over shared memory: lane
// (rg, cg) of a warp holds rows rg, rg + 8, ... and a group of columns, so operand rows come
// as broadcast 16-byte loads; every row is padded by 4 elements, which puts the 8 row groups
// on distinct banks.  In FP32, W3 stays in shared memory for the whole launch and W2 / W4 share
// a second buffer that is refilled by cp.async while the other layers compute.  The weight
// gradient of a tile is added into this CTA's slice of a partial buffer: the first tile
// stores, later tiles add with vector reductions (red.global.add) that the thread does not
// wait for.  Each element of a slice is written by one thread only, whose operations on it
// are applied in program order, so the sums are deterministic for a given grid.  The update
// kernel folds the slices in CTA order and applies Adam.
#include <cmath>

#include "pl_device.cuh"
#include "pl_kernels.h"
#include "pl_tcgen05.cuh"

namespace pl {

namespace {

constexpr int TR_THREADS = 256;
constexpr int NIN = 2;
// Blob offsets of the 2-input network: W1[64x2] b1 W2[128x64] b2 W3[128x128] b3 W4[64x128] b4 W5[3x64] b5.
constexpr int OW1 = 0, OB1 = OW1 + 64 * NIN, OW2 = OB1 + 64, OB2 = OW2 + 128 * 64, OW3 = OB2 + 128,
              OB3 = OW3 + 128 * 128, OW4 = OB3 + 128, OB4 = OW4 + 64 * 128, OW5 = OB4 + 64, OB5 = OW5 + 3 * 64,
              NPARAM = OB5 + 3;
static_assert(NPARAM == 33475, "blob of the 2-input network");
constexpr long long PSTRIDE = (NPARAM + 63) / 64 * 64;  // elements per CTA slice of the partials

template <typename R> struct TileOf;
template <> struct TileOf<float> { static constexpr int T = 16; static constexpr bool STAGE = true; };
template <> struct TileOf<double> { static constexpr int T = 8; static constexpr bool STAGE = false; };

constexpr int L64 = 64 + 4, L128 = 128 + 4;  // padded lengths of 64- and 128-wide rows
template <int K> struct Ld { static constexpr int v = K + 4; };

// Shared-memory plan (elements of R): activations of the 4 hidden layers [3T][N_l + 4], two
// reverse-pass buffers [3T][128 + 4], in FP32 the resident W3 [128][128 + 4] and the W2 / W4
// buffer [128][64 + 4] >= [64][128 + 4], and the per-sample scalars.
template <typename R>
struct Smem {
    static constexpr bool ST = TileOf<R>::STAGE;
    static constexpr int T = TileOf<R>::T, RT = 3 * T;
    static constexpr int A1 = 0, A2 = A1 + RT * L64, A3 = A2 + RT * L128, A4 = A3 + RT * L128, D0 = A4 + RT * L64,
                         D1 = D0 + RT * L128, WA = D1 + RT * L128, WB = WA + (ST ? 128 * L128 : 0),
                         X = WB + (ST ? 128 * L64 : 0), TG = X + 2 * T, O5 = TG + 3 * T, D5 = O5 + RT * 3,
                         IF = D5 + RT * 3, TOTAL = IF + T;
    static constexpr size_t bytes = (size_t)TOTAL * sizeof(R);
    static_assert(128 * L64 >= 64 * L128, "W2 / W4 buffer");
    static_assert(A2 % 4 == 0 && A3 % 4 == 0 && A4 % 4 == 0 && D0 % 4 == 0 && D1 % 4 == 0 && WA % 4 == 0 &&
                      WB % 4 == 0 && X % 4 == 0,
                  "16-byte aligned regions");
};
static_assert(Smem<float>::bytes <= 227 * 1024, "shared memory of one CTA");

template <typename R, int N>
__device__ __forceinline__ void ldv(const R* p, R (&v)[N]);
template <>
__device__ __forceinline__ void ldv<float, 4>(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ldv<float, 2>(const float* p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void ldv<double, 4>(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <>
__device__ __forceinline__ void ldv<double, 2>(const double* p, double (&v)[2]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    v[0] = a.x; v[1] = a.y;
}

template <typename R> __device__ __forceinline__ R tanh_r(R z);
template <> __device__ __forceinline__ float tanh_r<float>(float z) { return tanhf(z); }
template <> __device__ __forceinline__ double tanh_r<double>(double z) { return tanh(z); }
template <typename R> __device__ __forceinline__ R exp_r(R z);
template <> __device__ __forceinline__ float exp_r<float>(float z) { return expf(z); }
template <> __device__ __forceinline__ double exp_r<double>(double z) { return exp(z); }

// "g > threshold" with the decision an FP64 comparison gives (FP32 g: compare with the
// largest FP32 number not above the threshold).
__device__ __forceinline__ bool above(float g, double thr) { return g > __double2float_rd(thr); }
__device__ __forceinline__ bool above(double g, double thr) { return g > thr; }

// Partial-slice updates: the first tile stores, later tiles add.  FP32 adds are reductions
// the thread does not wait for; FP64 (the parity path) reads and writes.
__device__ __forceinline__ void acc1(float* p, float v, bool first) {
    if (first) *p = v;
    else asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}
__device__ __forceinline__ void acc1(double* p, double v, bool first) { *p = first ? v : *p + v; }
__device__ __forceinline__ void acc4(float* p, const float (&v)[4], bool first) {
    if (first) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]),
                     "f"(v[3])
                     : "memory");
}
__device__ __forceinline__ void acc4(double* p, const double (&v)[4], bool first) {
#pragma unroll
    for (int e = 0; e < 4; ++e) p[e] = first ? v[e] : p[e] + v[e];
}

// out[r][n] = sum_k in[r][k] W[n][k] (+ b[n] on the value rows r < T), n < NOUT.  Lane
// (rg, cg) = (lane / 4, lane % 4) of warp w computes rows rg + 8 i and columns
// w NOUT/8 + cg + 4 c.  Rows of `in` / `out` are padded (KIN + 4, NOUT + 4); rows of W have ldw.
template <typename R, int KIN, int NOUT>
__device__ __forceinline__ void dense_fwd(const R* in, const R* W, int ldw, const R* __restrict__ b, R* out) {
    constexpr int T = TileOf<R>::T, RPL = 3 * T / 8, CPL = NOUT / 32, LI = Ld<KIN>::v, LO = Ld<NOUT>::v;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, rg = lane >> 2, cg = lane & 3;
    const int nb = warp * (NOUT / 8) + cg;
    R acc[RPL][CPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[i][c] = R(0);
#pragma unroll 2
    for (int k = 0; k < KIN; k += 4) {
        R a[RPL][4], w[CPL][4];
#pragma unroll
        for (int i = 0; i < RPL; ++i) ldv<R, 4>(in + (rg + 8 * i) * LI + k, a[i]);
#pragma unroll
        for (int c = 0; c < CPL; ++c) ldv<R, 4>(W + (nb + 4 * c) * ldw + k, w[c]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < RPL; ++i)
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[i][c] = fma(a[i][q], w[c][q], acc[i][c]);
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int r = rg + 8 * i, n = nb + 4 * c;
            out[r * LO + n] = r < T ? acc[i][c] + b[n] : acc[i][c];
        }
}

// out[r][k] = sum_n dz[r][n] W[n][k], k < KIN (reverse pass of a dense layer).  Lane (rg, cg)
// of warp w computes rows rg + 8 i and the CPL = KIN/32 adjacent columns from
// w KIN/8 + cg CPL.
template <typename R, int KIN, int NOUT>
__device__ __forceinline__ void dense_bwd(const R* dz, const R* W, int ldw, R* out) {
    constexpr int T = TileOf<R>::T, RPL = 3 * T / 8, CPL = KIN / 32, LZ = Ld<NOUT>::v, LO = Ld<KIN>::v;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, rg = lane >> 2, cg = lane & 3;
    const int k0 = warp * (KIN / 8) + cg * CPL;
    R acc[RPL][CPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[i][c] = R(0);
#pragma unroll 2
    for (int n = 0; n < NOUT; n += 4) {
        R a[RPL][4];
#pragma unroll
        for (int i = 0; i < RPL; ++i) ldv<R, 4>(dz + (rg + 8 * i) * LZ + n, a[i]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            R w[CPL];
            ldv<R, CPL>(W + (n + q) * ldw + k0, w);
#pragma unroll
            for (int i = 0; i < RPL; ++i)
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[i][c] = fma(a[i][q], w[c], acc[i][c]);
        }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) out[(rg + 8 * i) * LO + k0 + c] = acc[i][c];
}

// Weight and bias gradient of a dense layer over the tile's rows, added to this CTA's slice:
// pw[n][k] += sum_r dz[r][n] in[r][k],  pb[n] += sum_{s < T} dz[s][n].  Warp w owns rows
// n of W in [w NOUT/8, (w+1) NOUT/8); lane = ng KG + kg holds 4 adjacent n and the column
// quads kg + KG j.
template <typename R, int KIN, int NOUT>
__device__ __forceinline__ void dense_wgrad(const R* dz, const R* in, R* pw, R* pb, bool first) {
    constexpr int T = TileOf<R>::T, RT = 3 * T, LZ = Ld<NOUT>::v, LI = Ld<KIN>::v;
    constexpr int NW = NOUT / 8, NG = NW / 4, KG = 32 / NG, KQ = KIN / (4 * KG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, ng = lane / KG, kg = lane % KG;
    const int n0 = warp * NW + 4 * ng;
    R acc[4][KQ][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < KQ; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = R(0);
#pragma unroll 2
    for (int r = 0; r < RT; ++r) {
        R d[4];
        ldv<R, 4>(dz + r * LZ + n0, d);
#pragma unroll
        for (int j = 0; j < KQ; ++j) {
            R a[4];
            ldv<R, 4>(in + r * LI + 4 * (kg + KG * j), a);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][j][e] = fma(d[i], a[e], acc[i][j][e]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < KQ; ++j) acc4(pw + (n0 + i) * KIN + 4 * (kg + KG * j), acc[i][j], first);
    if (threadIdx.x < NOUT) {
        R s = R(0);
        for (int q = 0; q < T; ++q) s += dz[q * LZ + threadIdx.x];
        acc1(pb + threadIdx.x, s, first);
    }
}

// Hidden activation in place: value rows z -> tanh(z), tangent rows z_d -> (1 - a^2) z_d.
template <typename R, int N>
__device__ __forceinline__ void tanh_fwd(R* A) {
    constexpr int T = TileOf<R>::T, L = Ld<N>::v, TL = T * L;
    for (int idx = threadIdx.x; idx < T * N; idx += TR_THREADS) {
        const int o = (idx / N) * L + idx % N;
        const R a = tanh_r<R>(A[o]), s = R(1) - a * a;
        A[o] = a;
        A[TL + o] *= s;
        A[2 * TL + o] *= s;
    }
}

// Reverse pass through a hidden activation: D holds dL/d(a, a_x, a_y), replaced by
// dL/d(z, z_x, z_y); A holds (a, a_x, a_y).
template <typename R, int N>
__device__ __forceinline__ void tanh_bwd(const R* A, R* D) {
    constexpr int T = TileOf<R>::T, L = Ld<N>::v, TL = T * L;
    for (int idx = threadIdx.x; idx < T * N; idx += TR_THREADS) {
        const int o = (idx / N) * L + idx % N;
        const R a = A[o], ax = A[TL + o], ay = A[2 * TL + o], s = R(1) - a * a;
        const R d0 = D[o], d1 = D[TL + o], d2 = D[2 * TL + o];
        D[o] = s * d0 - R(2) * a * (ax * d1 + ay * d2);
        D[TL + o] = s * d1;
        D[2 * TL + o] = s * d2;
    }
}

// Asynchronous copy of W[N][K] (FP32 master weights) into padded shared rows (K + 4); the
// caller waits with stage_wait() and a barrier before reading.
template <int N, int K>
__device__ __forceinline__ void stage_async(const float* __restrict__ w, float* ws) {
    for (int i = threadIdx.x; i < N * K / 4; i += TR_THREADS) {
        const int n = i / (K / 4), k4 = i % (K / 4);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(ws + n * (K + 4) + 4 * k4);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(__cvta_generic_to_global(w + n * K + 4 * k4))
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Loss terms of one sample and dL/d(outputs) for its value and tangent rows.
template <typename R>
struct SampleLoss {
    R g[3], gx[3], gy[3];
    R ld, lp, li;   // the sample's terms (squares summed in R)
};

template <typename R>
__device__ __forceinline__ SampleLoss<R> sample_loss(const R (&o)[3], const R (&ox)[3], const R (&oy)[3],
                                                     const R (&t)[3], bool iface, R sx, R sy, R inv_n, R c_phys,
                                                     R c_int, const TrainLat& L, const TrainHyper& hp) {
    SampleLoss<R> q;
    const R r = o[0], u = o[1], v = o[2];
    const R rx = sx * ox[0], ux = sx * ox[1], vx = sx * ox[2];
    const R ry = sy * oy[0], uy = sy * oy[1], vy = sy * oy[2];
    // Eq. 4
    R e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e[k] = o[k] - t[k];
        q.g[k] = R(2) * e[k] * inv_n;
    }
    q.ld = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    // Eqs. 5-7: p' and p'' of p = rho/3 + G psi^2/6
    const R rho0 = R(L.rho0), G = R(L.G);
    const R ex = exp_r<R>(-r / rho0), psi = rho0 * (R(1) - ex);
    const R P = R(1) / R(3) + G * psi * ex / R(3);
    const R dP = G * (ex * ex - psi * ex / rho0) / R(3);
    const R rc = u * rx + r * ux + v * ry + r * vy;
    const R rmx = u * u * rx + R(2) * r * u * ux + u * v * ry + r * v * uy + r * u * vy + P * rx;
    const R rmy = u * v * rx + r * v * ux + r * u * vx + v * v * ry + R(2) * r * v * vy + P * ry;
    q.lp = rc * rc + rmx * rmx + rmy * rmy;
    const R A = c_phys * rc, B = c_phys * rmx, C = c_phys * rmy;
    const R dr = A * (ux + vy) + B * (R(2) * u * ux + v * uy + u * vy + dP * rx) +
                 C * (v * ux + u * vx + R(2) * v * vy + dP * ry);
    const R du = A * rx + B * (R(2) * u * rx + R(2) * r * ux + v * ry + r * vy) + C * (v * rx + r * vx);
    const R dv = A * ry + B * (u * ry + r * uy) + C * (u * rx + r * ux + R(2) * v * ry + R(2) * r * vy);
    R drx = A * u + B * (u * u + P) + C * (u * v);
    R dry = A * v + B * (u * v) + C * (v * v + P);
    const R dux = A * r + B * (R(2) * r * u) + C * (r * v);
    const R duy = B * (r * v);
    const R dvx = C * (r * u);
    const R dvy = A * r + B * (r * u) + C * (R(2) * r * v);
    // Eq. 8 (signs of the text)
    q.li = R(0);
    if (iface) {
        const R qq = rx * rx + ry * ry;
        const R a1 = R(hp.alpha1), a2 = R(hp.alpha2);
        q.li = -a1 * qq + a2 * qq * qq;
        const R dq = c_int * (-a1 + R(2) * a2 * qq);
        drx += R(2) * dq * rx;
        dry += R(2) * dq * ry;
    }
    q.g[0] += dr;
    q.g[1] += du;
    q.g[2] += dv;
    q.gx[0] = sx * drx; q.gx[1] = sx * dux; q.gx[2] = sx * dvx;
    q.gy[0] = sy * dry; q.gy[1] = sy * duy; q.gy[2] = sy * dvy;
    return q;
}

template <typename R>
__global__ void __launch_bounds__(TR_THREADS, 1)
k_train_grad(TrainLat L, const R* __restrict__ w, R* __restrict__ part, double* __restrict__ loss_part,
             const unsigned long long* __restrict__ ni_dev, TrainHyper hp, long long ntiles) {
    using SM = Smem<R>;
    constexpr int T = SM::T, RT = SM::RT;
    constexpr bool ST = TileOf<R>::STAGE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    R *A1 = sm + SM::A1, *A2 = sm + SM::A2, *A3 = sm + SM::A3, *A4 = sm + SM::A4;
    R *D0 = sm + SM::D0, *D1 = sm + SM::D1, *X = sm + SM::X, *TG = sm + SM::TG;
    R *O5 = sm + SM::O5, *D5 = sm + SM::D5, *IF = sm + SM::IF;
    const int tid = threadIdx.x;
    if ((long long)blockIdx.x >= ntiles) return;   // no tile, no slice (the fold skips it)
    const long long N = (long long)L.nx * L.ny;
    const unsigned long long ni = *ni_dev;
    const R sx = R(2.0 / L.nx), sy = R(2.0 / L.ny), inv_n = R(1.0 / (double)N);
    const R c_phys = R(2.0 * hp.lambda_phys / (double)N);
    const R c_int = ni ? R(hp.lambda_int / (double)ni) : R(0);
    const R* rho = static_cast<const R*>(L.rho);
    const R* jx = static_cast<const R*>(L.jx);
    const R* jy = static_cast<const R*>(L.jy);
    const R* gf = static_cast<const R*>(L.g);
    R* P = part + (long long)blockIdx.x * PSTRIDE;
    double ld = 0.0, lp = 0.0, li = 0.0;
    // Weight operands: FP32 reads W3 from its resident copy and W2 / W4 from the shared buffer
    // WB (W2 on entry to every tile); FP64 reads the master weights in place.
    const R* W2 = w + OW2;
    const R* W3 = w + OW3;
    const R* W4 = w + OW4;
    int ld2 = 64, ld3 = 128, ld4 = 128;
    if constexpr (ST) {
        R* WA = sm + SM::WA;
        R* WB = sm + SM::WB;
        stage_async<128, 128>(w + OW3, WA);
        stage_async<128, 64>(w + OW2, WB);
        stage_wait();
        W2 = WB; W3 = WA; W4 = WB;
        ld2 = L64; ld3 = L128; ld4 = L128;
    }
    __syncthreads();

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;
        if (tid < T) {
            const long long c = tile * T + tid;
            const bool valid = c < N;
            const long long cc = valid ? c : N - 1;
            const int x = (int)(cc % L.nx), y = (int)(cc / L.nx);
            X[2 * tid] = R(2) * (R(x) + R(0.5)) / R(L.nx) - R(1);
            X[2 * tid + 1] = R(2) * (R(y) + R(0.5)) / R(L.ny) - R(1);
            const R r = rho[cc];
            TG[3 * tid] = r;
            TG[3 * tid + 1] = jx[cc] / r;
            TG[3 * tid + 2] = jy[cc] / r;
            IF[tid] = valid ? (above(gf[cc], L.threshold) ? R(1) : R(0)) : R(-1);  // -1: padding sample
        }
        __syncthreads();
        // layer 1 (2 -> 64): value rows from (x^, y^), tangent rows are W1's columns
        for (int idx = tid; idx < RT * 64; idx += TR_THREADS) {
            const int r = idx / 64, n = idx % 64, ch = r / T, s = r % T;
            const R w0 = w[OW1 + 2 * n], w1 = w[OW1 + 2 * n + 1];
            A1[r * L64 + n] = ch == 0 ? X[2 * s] * w0 + X[2 * s + 1] * w1 + w[OB1 + n] : (ch == 1 ? w0 : w1);
        }
        __syncthreads();
        tanh_fwd<R, 64>(A1);
        __syncthreads();
        dense_fwd<R, 64, 128>(A1, W2, ld2, w + OB2, A2);               // layer 2 (W2 in WB)
        __syncthreads();
        if constexpr (ST) stage_async<64, 128>(w + OW4, sm + SM::WB);   // W4 -> WB behind layer 3
        tanh_fwd<R, 128>(A2);
        __syncthreads();
        dense_fwd<R, 128, 128>(A2, W3, ld3, w + OB3, A3);              // layer 3
        if constexpr (ST) stage_wait();
        __syncthreads();
        tanh_fwd<R, 128>(A3);
        __syncthreads();
        dense_fwd<R, 128, 64>(A3, W4, ld4, w + OB4, A4);               // layer 4 (W4 in WB)
        __syncthreads();
        tanh_fwd<R, 64>(A4);
        __syncthreads();
        // layer 5 (64 -> 3, linear)
        for (int idx = tid; idx < RT * 3; idx += TR_THREADS) {
            const int r = idx / 3, o = idx % 3;
            R acc = R(0);
            for (int k = 0; k < 64; ++k) acc = fma(A4[r * L64 + k], w[OW5 + o * 64 + k], acc);
            O5[idx] = r < T ? acc + w[OB5 + o] : acc;
        }
        __syncthreads();
        // loss and dL/d(outputs), rows s, T + s, 2T + s
        if (tid < T) {
            const int s = tid;
            if (IF[s] >= R(0)) {
                const R o[3] = {O5[3 * s], O5[3 * s + 1], O5[3 * s + 2]};
                const R ox[3] = {O5[3 * (T + s)], O5[3 * (T + s) + 1], O5[3 * (T + s) + 2]};
                const R oy[3] = {O5[3 * (2 * T + s)], O5[3 * (2 * T + s) + 1], O5[3 * (2 * T + s) + 2]};
                const R t[3] = {TG[3 * s], TG[3 * s + 1], TG[3 * s + 2]};
                const SampleLoss<R> q = sample_loss<R>(o, ox, oy, t, IF[s] > R(0), sx, sy, inv_n, c_phys, c_int, L, hp);
                ld += q.ld;
                lp += q.lp;
                li += q.li;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    D5[3 * s + k] = q.g[k];
                    D5[3 * (T + s) + k] = q.gx[k];
                    D5[3 * (2 * T + s) + k] = q.gy[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) D5[3 * s + k] = D5[3 * (T + s) + k] = D5[3 * (2 * T + s) + k] = R(0);
            }
        }
        __syncthreads();
        // layer 5 reverse: dW5, db5 and dL/dA4 -> D0 [3T][64]
        for (int idx = tid; idx < 3 * 64; idx += TR_THREADS) {
            const int o = idx / 64, k = idx % 64;
            R acc = R(0);
            for (int r = 0; r < RT; ++r) acc = fma(D5[3 * r + o], A4[r * L64 + k], acc);
            acc1(P + OW5 + idx, acc, first);
        }
        if (tid >= 192 && tid < 195) {
            const int o = tid - 192;
            R acc = R(0);
            for (int s = 0; s < T; ++s) acc += D5[3 * s + o];
            acc1(P + OB5 + o, acc, first);
        }
        for (int idx = tid; idx < RT * 64; idx += TR_THREADS) {
            const int r = idx / 64, k = idx % 64;
            D0[r * L64 + k] =
                D5[3 * r] * w[OW5 + k] + D5[3 * r + 1] * w[OW5 + 64 + k] + D5[3 * r + 2] * w[OW5 + 128 + k];
        }
        __syncthreads();
        tanh_bwd<R, 64>(A4, D0);
        __syncthreads();
        // layer 4 (128 -> 64), W4 in WB
        dense_wgrad<R, 128, 64>(D0, A3, P + OW4, P + OB4, first);
        dense_bwd<R, 128, 64>(D0, W4, ld4, D1);
        __syncthreads();
        if constexpr (ST) stage_async<128, 64>(w + OW2, sm + SM::WB);   // W2 -> WB behind layer 3
        tanh_bwd<R, 128>(A3, D1);
        __syncthreads();
        // layer 3 (128 -> 128)
        dense_wgrad<R, 128, 128>(D1, A2, P + OW3, P + OB3, first);
        dense_bwd<R, 128, 128>(D1, W3, ld3, D0);
        if constexpr (ST) stage_wait();
        __syncthreads();
        tanh_bwd<R, 128>(A2, D0);
        __syncthreads();
        // layer 2 (64 -> 128), W2 in WB (and for the next tile's forward pass)
        dense_wgrad<R, 64, 128>(D0, A1, P + OW2, P + OB2, first);
        dense_bwd<R, 64, 128>(D0, W2, ld2, D1);
        __syncthreads();
        tanh_bwd<R, 64>(A1, D1);
        __syncthreads();
        // layer 1 (2 -> 64): inputs (x^, y^) on the value rows, unit vectors on the tangent rows
        if (tid < 64) {
            R s0 = R(0), s1 = R(0), sb = R(0);
            for (int s = 0; s < T; ++s) {
                const R d0 = D1[s * L64 + tid], d1 = D1[(T + s) * L64 + tid], d2 = D1[(2 * T + s) * L64 + tid];
                s0 += d0 * X[2 * s] + d1;
                s1 += d0 * X[2 * s + 1] + d2;
                sb += d0;
            }
            acc1(P + OW1 + 2 * tid, s0, first);
            acc1(P + OW1 + 2 * tid + 1, s1, first);
            acc1(P + OB1 + tid, sb, first);
        }
        __syncthreads();
    }
    double v[3] = {ld, lp, li};
    const int op[3] = {0, 0, 0};
    block_reduce<3>(v, op, reinterpret_cast<double*>(D0));   // D0 is free here
    if (tid == 0)
        for (int k = 0; k < 3; ++k) loss_part[blockIdx.x * 4 + k] = v[k];
}

// Interface-cell count (exact integer sum) and the master weights from the FP32 blob.
template <typename R>
__global__ void k_train_prep(TrainLat L, const float* __restrict__ w32, R* __restrict__ master,
                             unsigned long long* __restrict__ ni) {
    const long long N = (long long)L.nx * L.ny;
    const R* g = static_cast<const R*>(L.g);
    unsigned cnt = 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        cnt += above(g[c], L.threshold) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(ni, (unsigned long long)cnt);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPARAM; p += gridDim.x * blockDim.x) master[p] = R(w32[p]);
}

// Fold the CTA slices (CTA order), keep the gradient, apply Adam if `apply`; block 0 also
// folds the loss terms into hist_row = (L, L_data, L_phys, L_int).
template <typename R>
__global__ void k_train_update(R* __restrict__ master, R* __restrict__ m, R* __restrict__ v, R* __restrict__ grad,
                               const R* __restrict__ part, const double* __restrict__ loss_part,
                               const unsigned long long* __restrict__ ni, int nact, long long ncells,
                               TrainHyper hp, double bc1, double bc2, int apply, double* __restrict__ hist_row) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPARAM; p += gridDim.x * blockDim.x) {
        SumAcc<R> acc;
        for (int b = 0; b < nact; ++b) acc.add(part[(long long)b * PSTRIDE + p]);
        const R g = R(acc.value());
        grad[p] = g;
        if (apply) {
            const R mm = R(hp.beta1) * m[p] + R(1.0 - hp.beta1) * g;
            const R vv = R(hp.beta2) * v[p] + R(1.0 - hp.beta2) * g * g;
            m[p] = mm;
            v[p] = vv;
            master[p] -= R(hp.lr) * (mm * R(bc1)) / (sqrt(vv * R(bc2)) + R(hp.eps));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < nact; ++b)
            for (int k = 0; k < 3; ++k) s[k] += loss_part[b * 4 + k];
        const double Ld = s[0] / (double)ncells, Lp = s[1] / (double)ncells;
        const double Li = *ni ? s[2] / (double)*ni : 0.0;
        hist_row[0] = Ld + hp.lambda_phys * Lp + hp.lambda_int * Li;
        hist_row[1] = Ld;
        hist_row[2] = Lp;
        hist_row[3] = Li;
    }
}

template <typename R>
__global__ void k_train_finish(const R* __restrict__ master, float* __restrict__ w32) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPARAM; p += gridDim.x * blockDim.x)
        w32[p] = (float)master[p];
}

constexpr int UPD_GRID = 132, UPD_THREADS = 256;  // 33,792 threads >= one per parameter

template <typename R>
cudaError_t grad_setup(int* grid) {
    static int g_grid = 0;  // per process and instantiation (one device)
    if (!g_grid) {
        cudaError_t e = cudaFuncSetAttribute(k_train_grad<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Smem<R>::bytes);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_train_grad<R>, TR_THREADS, Smem<R>::bytes)) !=
            cudaSuccess)
            return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        g_grid = sms * occ;
    }
    *grid = g_grid;
    return cudaSuccess;
}


// ---------------------------------------------------------------------------------------------
// Tensor-core form: the dense layers 2-4 of the forward pass, of the reverse pass and of the
// weight gradient, and the bias and layer-1 gradients, as tcgen05 MMAs (BF16 operands in shared
// memory, FP32 accumulators in TMEM); the layer-1 forward pass, layer 5, the loss and the tanh
// terms on CUDA cores in FP32.
//
// Sixteen warps per CTA (one CTA per SM: all of TMEM).  A tile is 40 samples as 128 operand
// rows: row 32 u + 3 q + c is channel c (value, d/dx^, d/dy^) of sample 10 u + q; lanes 30 and
// 31 of each warp are padding (zero rows).  Warp w serves TMEM lane quadrant u = w mod 4 (thread
// r owns row r, i.e. TMEM lane r) and the 16-column chunks 16 (w / 4) + 64 i.  The three rows of
// a sample are neighbouring lanes of one warp, so the tanh terms that couple them (s = 1 - a^2 for
// the tangent rows, the second-derivative term of the value row) move by warp shuffles.  Every
// activation is stored once, K-major over its features: it is the A operand of the next forward
// MMA and, read MN-major (K = rows), an operand of the gradient MMAs; the weight images serve the
// forward MMAs K-major and the reverse MMAs MN-major (K = outputs).  In the reverse pass dZ_l
// (l = 3, 2, 1) overwrites A_l once the MMAs that read A_l are complete.
//   forward   Z_l = A_{l-1} W_l^T                               M = 128 rows, N = out_l, K = in_l
//   reverse   dA_{l-1} = dZ_l W_l                                M = 128 rows, N = in_l,  K = out_l
//   gradient  [. . db_2 | dW_2] += dZ_2^T [E_1 | A_1]            M = out_2, N = 16 + in_2, K = 128 rows
//             [dW_3 | . . db_3] += dZ_3^T [A_2 | E_2]            M = out_3, N = in_3 + 16, K = 128 rows
//             dW_4^T += A_3^T dZ_4                                M = in_4,  N = out_4,     K = 128 rows
//             [dW_1 | db_1 ; . . db_4] += [dZ_1 | dZ_4]^T E_1     M = 64 + 64, N = 16,      K = 128 rows
// E_1, 16 columns stored just before A1, holds per row (x^, y^, 1) on value rows, (1, 0, 0) on
// d/dx^ rows and (0, 1, 0) on d/dy^ rows, zeros elsewhere, so that dZ_1^T E_1 gives the layer-1
// gradient (columns 0 and 1: the sums of dz_v x^ + dz_x and dz_v y^ + dz_y; column 2: of dz_v);
// its column 2, the value-row indicator, gives the bias gradients of the layers above.  E_2, the 16
// columns after A2's features, holds the indicator in its column 2 as well.  dZ_4 has a buffer of
// its own right after A1 (A4 stays readable for the layer-5 gradient meanwhile), so that the
// last row is one M = 128 MMA.  Everything
// accumulates in TMEM over the CTA's tiles and is written once; layer 5 goes to the CTA's
// partial slice per tile, as in the FP32 kernel.
namespace ttc {
constexpr int THREADS = 512;                       // four warps per TMEM lane quadrant
constexpr int NH = THREADS / 128;                  // warps per quadrant: warp w takes the column
constexpr int CS = 16 * NH;                        // chunks 16 (w / 4) + CS i of 16 columns
constexpr int SPT = 40;                            // samples per tile
constexpr int COLB = 128 * 2;                      // bytes of one feature of a 128-row BF16 operand
constexpr int OFF_E1 = 0, OFF_A1 = OFF_E1 + 16 * COLB, OFF_DZ4 = OFF_A1 + 64 * COLB, OFF_A4 = OFF_DZ4 + 64 * COLB,
              OFF_A2 = OFF_A4 + 64 * COLB,
              OFF_E2 = OFF_A2 + 128 * COLB, OFF_A3 = OFF_E2 + 16 * COLB, OFF_W2 = OFF_A3 + 128 * COLB,
              OFF_W3 = OFF_W2 + 128 * 64 * 2, OFF_W4 = OFF_W3 + 128 * 128 * 2, OFF_SC = OFF_W4 + 64 * 128 * 2;
// FP32 scratch: dL/d(outputs) per row [128][4]; the layer-5 partial sums of the warps with
// w / 4 > 0 [NH - 1][128][4]; the layer-5 gradient partials [8][GP_LD] (lane l's 24 at l * 25)
constexpr int GP_LD = 32 * 25 + 8;                 // 808 = 8 mod 32: the fold reads distinct banks
constexpr int OFF_S5 = OFF_SC, OFF_X = OFF_S5 + 128 * 4 * 4, OFF_GP = OFF_X + (NH - 1) * 128 * 4 * 4,
              OFF_PAR = OFF_GP + 8 * GP_LD * 4, OFF_BAR = OFF_PAR + 704 * 4, OFF_SLOT = OFF_BAR + 16,
              SMEM = OFF_SLOT + 16;
// FP32 parameters kept in shared memory (floats from OFF_PAR): b1, b2, b3, b4, W5, then W1 by
// column (W1[k][0] at PW1 + k, W1[k][1] at PW1 + 64 + k)
constexpr int PB1 = 0, PB2 = 64, PB3 = 192, PB4 = 320, PW5 = 384, PW1 = 576, NPAR = 704;
static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
static_assert(OFF_PAR % 16 == 0 && OFF_W2 % 16 == 0, "16-byte aligned regions");
static_assert(OFF_A1 == OFF_E1 + 2 * 2048 && OFF_DZ4 == OFF_A1 + 8 * 2048 && OFF_E2 == OFF_A2 + 16 * 2048,
              "operands read as one: [E1 | A1], [A1 | DZ4], [A2 | E2]");
constexpr int WIMG_BYTES = (128 * 64 + 128 * 128 + 64 * 128) * 2;   // W2, W3, W4 at the head of the image
// TMEM columns (each accumulator 32-column aligned): work 128, [db2 | dW2] 80, [dW3 | db3] 144,
// dW4^T 64, [dW1 | db1 ; db4] 16
constexpr uint32_t TM_WORK = 0, TM_DW2 = 128, TM_DW3 = 224, TM_DW4T = 384, TM_D1 = 448, TM_COLS = 512;
static_assert(TM_DW2 + 80 <= TM_DW3 && TM_DW3 + 144 <= TM_DW4T && TM_DW4T + 64 <= TM_D1 && TM_D1 + 16 <= TM_COLS,
              "TMEM columns");
constexpr uint32_t KLBO = 2048;                    // K-major 128-row operand: core matrices along K

// D (+)= A B over K in steps of 16 (each operand: base address, leading and stride byte
// offsets, byte step per K step, major).
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, uint32_t alb, uint32_t asb, uint32_t ast,
                                          bool amn, uint32_t b, uint32_t blb, uint32_t bsb, uint32_t bst, bool bmn,
                                          int N, int K, bool acc) {
    const uint32_t idesc = tc::idesc_bf16(128, N, amn, bmn);
    // the start address is the descriptor's low field (address >> 4; every operand lies below
    // 256 KB, so the field never carries): a K step adds step >> 4
    uint64_t da = tc::smem_desc(a, alb, asb), db = tc::smem_desc(b, blb, bsb);
    for (int ks = 0; ks < K / 16; ++ks) {
        tc::mma_bf16(d, da, db, idesc, (acc || ks > 0) ? 1u : 0u);
        da += ast >> 4;
        db += bst >> 4;
    }
}
// D (+)= A^T B with both operands 128-row activation buffers read MN-major (K = the 128 rows)
__device__ __forceinline__ void mma_rows(uint32_t d, uint32_t a, uint32_t b, int N, bool acc) {
    mma_chain(d, a, 128, KLBO, 256, true, b, 128, KLBO, 256, true, N, 128, acc);
}

// 8 BF16 values of row r, features k0..k0+7, of a K-major 128-row operand -> FP32.
__device__ __forceinline__ void load8(const uint8_t* A, int r, int k0, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(A + ((k0 >> 3) * 16 + (r >> 3)) * 128 + (r & 7) * 16);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[q]));
        v[2 * q] = f.x;
        v[2 * q + 1] = f.y;
    }
}

using tc::add2;   // packed FP32 pairs (f32x2)
using tc::bc2;
using tc::fma2;
using tc::ld2;
using tc::mul2;
using tc::sub2;

// Row roles of thread r; kv = 1 on value rows, kt = 1 on tangent rows (both 0 on padding rows).
struct Row {
    int r, lane, warp, c;
    bool pad;
    float kv, kt;
};

// Forward epilogue of a hidden layer from 16 pre-activations z (bias added on value rows):
// value rows a = tanh(z), tangent rows (1 - a^2) z with a of their sample; out = FP32 values.
__device__ __forceinline__ void act16(const Row& R, const float* __restrict__ b, int c0, const float (&z)[16],
                                      float (&out)[16]) {
    const float2 kv = bc2(R.kv), kt = bc2(R.kt), one = bc2(1.0f);
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const float2 zz = fma2(kv, ld2(b + c0 + j), make_float2(z[j], z[j + 1]));
        const float2 a = make_float2(tc::tanh_fast(zz.x), tc::tanh_fast(zz.y));
        const float2 sg = sub2(one, mul2(a, a));
        const float2 sv = make_float2(__shfl_sync(0xffffffffu, sg.x, R.lane - R.c),
                                      __shfl_sync(0xffffffffu, sg.y, R.lane - R.c));
        const float2 o = fma2(kt, mul2(sv, zz), mul2(kv, a));
        out[j] = o.x;
        out[j + 1] = o.y;
    }
}

// Reverse pass through a hidden activation for 16 features: dA (this row's dL/d act) -> dL/dz.
// av / own: the stored activations of the sample's value row and of this row.  Value rows:
// s dA - 2 a (a_x dA_x + a_y dA_y); tangent rows: s dA_d; s = 1 - a^2 of the sample.  Each
// tangent row forms its product a_d dA_d, which the value row takes from the next two lanes.
__device__ __forceinline__ void dact16(const Row& R, const float (&dA)[16], const float (&av)[16],
                                       const float (&own)[16], float (&dz)[16]) {
    const float2 m = bc2(-2.0f * R.kv), one = bc2(1.0f);
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const float2 d = make_float2(dA[j], dA[j + 1]), a = make_float2(av[j], av[j + 1]);
        const float2 p = mul2(make_float2(own[j], own[j + 1]), d);
        const float2 px = make_float2(__shfl_sync(0xffffffffu, p.x, R.lane + 1),
                                      __shfl_sync(0xffffffffu, p.y, R.lane + 1));
        const float2 py = make_float2(__shfl_sync(0xffffffffu, p.x, R.lane + 2),
                                      __shfl_sync(0xffffffffu, p.y, R.lane + 2));
        const float2 sg = sub2(one, mul2(a, a));
        const float2 o = fma2(mul2(m, a), add2(px, py), mul2(sg, d));
        dz[j] = o.x;
        dz[j + 1] = o.y;
    }
}

// 16 stored activations (features c0..c0+15) of row r.
__device__ __forceinline__ void load16(const uint8_t* A, int r, int c0, float (&v)[16]) {
    float t[8];
    load8(A, r, c0, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = t[j];
    load8(A, r, c0 + 8, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[8 + j] = t[j];
}

// The activations of this row's sample's value row and of this row (both in the warp's own
// quadrant, so that a warp may overwrite its rows' chunk in place).
__device__ __forceinline__ void sample_acts(const Row& R, const uint8_t* A, int c0, float (&av)[16], float (&own)[16]) {
    load16(A, R.r - R.c, c0, av);
    load16(A, R.r, c0, own);
}

__device__ __forceinline__ void store16(uint8_t* A, int r, int c0, const float (&v)[16]) {
    tc::store8(A, r, c0, v);
    tc::store8(A, r, c0 + 8, v + 8);
}
}  // namespace ttc

__global__ void __launch_bounds__(ttc::THREADS, 1)
k_train_grad_tc(TrainLat L, const float* __restrict__ w, const uint16_t* __restrict__ wimg, float* __restrict__ part,
                double* __restrict__ loss_part, const unsigned long long* __restrict__ ni_dev, TrainHyper hp,
                long long ntiles, unsigned* __restrict__ err) {
    using namespace ttc;
    extern __shared__ __align__(1024) uint8_t sm[];
    if ((long long)blockIdx.x >= ntiles) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int h = warp >> 2;   // column group: this warp takes the 16-column chunks 16 h, 16 h + CS, ...
    Row R;
    R.lane = tid & 31;
    R.warp = warp & 3;         // TMEM lane quadrant
    R.r = 32 * R.warp + R.lane;
    R.c = R.lane % 3;
    R.pad = R.lane >= 30;
    R.kv = (!R.pad && R.c == 0) ? 1.0f : 0.0f;
    R.kt = (!R.pad && R.c != 0) ? 1.0f : 0.0f;
    const int q = R.lane / 3;
    uint8_t *E1 = sm + OFF_E1, *A1 = sm + OFF_A1, *A2 = sm + OFF_A2, *A3 = sm + OFF_A3, *A4 = sm + OFF_A4,
            *DZ4 = sm + OFF_DZ4;
    float* S5 = reinterpret_cast<float*>(sm + OFF_S5);
    float* X = reinterpret_cast<float*>(sm + OFF_X);
    float* GP = reinterpret_cast<float*>(sm + OFF_GP);
    float* PAR = reinterpret_cast<float*>(sm + OFF_PAR);
    for (int i = tid; i < NPAR; i += THREADS)
        PAR[i] = i < PB2 ? w[OB1 + i] : (i < PB3 ? w[OB2 + i - PB2] : (i < PB4 ? w[OB3 + i - PB3] :
                 (i < PW5 ? w[OB4 + i - PB4] : (i < PW1 ? w[OW5 + i - PW5] :
                 w[OW1 + 2 * ((i - PW1) % 64) + (i - PW1) / 64]))));
    if (h == 0) {   // E2: the value-row indicator in column 2 (the same for every tile)
        float e[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) e[j] = 0.0f;
        e[2] = (R.c == 0 && !R.pad) ? 1.0f : 0.0f;
        store16(A2, R.r, 128, e);
    }
    const uint32_t bar_w = tc::saddr(sm + OFF_BAR), bar_mma = tc::saddr(sm + OFF_BAR + 8);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
    if (tid == 0) {
        tc::mbar_init(bar_w, 1);
        tc::mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(slot)),
                     "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_before_sync();
    __syncthreads();
    tc::tc_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lane_off = (uint32_t)(32 * R.warp) << 16;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w), "r"(WIMG_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::saddr(sm + OFF_W2)),
                     "l"(wimg), "r"(WIMG_BYTES), "r"(bar_w)
                     : "memory");
    }
    bool ok = __syncthreads_and(tc::mbar_wait(bar_w, 0)) != 0;
    uint32_t phase = 0;
    bool pending = false;
    const long long N = (long long)L.nx * L.ny;
    const unsigned long long ni = *ni_dev;
    const float sx = 2.0f / (float)L.nx, sy = 2.0f / (float)L.ny, inv_n = (float)(1.0 / (double)N);
    const float c_phys = (float)(2.0 * hp.lambda_phys / (double)N);
    const float c_int = ni ? (float)(hp.lambda_int / (double)ni) : 0.0f;
    const float* rho = static_cast<const float*>(L.rho);
    const float* jx = static_cast<const float*>(L.jx);
    const float* jy = static_cast<const float*>(L.jy);
    const float* gf = static_cast<const float*>(L.g);
    float* P = part + (long long)blockIdx.x * PSTRIDE;
    // loss terms: FP32 per thread (a few dozen samples each), FP64 from the CTA reduction on
    float ld = 0.0f, lp = 0.0f, li = 0.0f;
    const float thr = __double2float_rd(L.threshold);   // g > thr, as in above()
    const uint32_t sE1 = tc::saddr(E1), sA1 = tc::saddr(A1), sA2 = tc::saddr(A2), sA3 = tc::saddr(A3),
                   sDZ4 = tc::saddr(DZ4), sW2 = tc::saddr(sm + OFF_W2), sW3 = tc::saddr(sm + OFF_W3),
                   sW4 = tc::saddr(sm + OFF_W4);

    // operands written by the threads -> visible to the tensor core, then thread 0 issues
    auto sync_to_mma = [&]() {
        tc::fence_async_smem();
        tc::tc_before_sync();
        __syncthreads();
        tc::tc_after_sync();
        return ok;
    };
    // wait (bounded) for the last commit to bar_mma; false on timeout
    auto wait_issued = [&]() {
        pending = true;
        ok = __syncthreads_and(tc::mbar_wait(bar_mma, phase)) != 0;
        if (ok) {
            pending = false;
            phase ^= 1;
        }
        tc::tc_after_sync();
        return ok;
    };
    // commit the issued MMAs and wait for them
    auto wait_mma = [&]() {
        if (tid == 0) tc::mma_commit(bar_mma);
        return wait_issued();
    };

    for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;
        const long long smp = tile * SPT + R.warp * 10 + q;
        const bool valid = !R.pad && smp < N;
        const long long cc = valid ? smp : 0;
        int x, y;
        if (N <= 0xffffffffLL) {   // 32-bit division (every lattice of practical size)
            const unsigned c32 = (unsigned)cc, q32 = c32 / (unsigned)L.nx;
            x = (int)(c32 - q32 * (unsigned)L.nx);
            y = (int)q32;
        } else {
            x = (int)(cc % L.nx);
            y = (int)(cc / L.nx);
        }
        // the loss targets of the value rows, loaded now so that their latency is hidden by the
        // forward pass
        float t_rho = 1.0f, t_jx = 0.0f, t_jy = 0.0f, t_g = 0.0f;
        if (h == 0 && valid && R.c == 0) {
            t_rho = rho[cc];
            t_jx = jx[cc];
            t_jy = jy[cc];
            t_g = gf[cc];
        }
        const float xh = 2.0f * ((float)x + 0.5f) / (float)L.nx - 1.0f;
        const float yh = 2.0f * ((float)y + 0.5f) / (float)L.ny - 1.0f;

        // ---- layer 1 (2 -> 64) on CUDA cores: value rows from (x^, y^), tangent rows W1's columns;
        // this warp's chunk (64 = CS columns: one) in registers first
        static_assert(CS == 64, "layer 1: one 16-column chunk per warp");
        const int c1 = 16 * h;
        const float2 cx = bc2(R.c == 0 ? xh : (R.c == 1 ? 1.0f : 0.0f));   // value rows (x^, y^), tangent
        const float2 cy = bc2(R.c == 0 ? yh : (R.c == 2 ? 1.0f : 0.0f));   // rows the unit vectors
        float a1[16];
        {
            float z[16];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float2 zz = fma2(cx, ld2(PAR + PW1 + c1 + j), mul2(cy, ld2(PAR + PW1 + 64 + c1 + j)));
                z[j] = zz.x;
                z[j + 1] = zz.y;
            }
            act16(R, PAR + PB1, c1, z, a1);
        }
        // the previous tile's gradient MMA reads E1 and A1: complete before they are rewritten
        if (pending && !wait_issued()) break;
        if (h == 0) {   // E1 of this row (samples past the lattice end have dZ = 0: any finite entry)
            float e[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) e[j] = 0.0f;
            if (!R.pad) {
                e[0] = R.c == 0 ? xh : (R.c == 1 ? 1.0f : 0.0f);
                e[1] = R.c == 0 ? yh : (R.c == 2 ? 1.0f : 0.0f);
                e[2] = R.c == 0 ? 1.0f : 0.0f;
            }
            store16(E1, R.r, 0, e);
        }
        store16(A1, R.r, c1, a1);
        // ---- layers 2-4: MMA, then the activation epilogue (layer 4 also feeds layer 5)
        float2 o2[3] = {bc2(0.0f), bc2(0.0f), bc2(0.0f)};
#pragma unroll 1
        for (int layer = 2; layer <= 4 && ok; ++layer) {
            if (!sync_to_mma()) break;
            const int Nout = layer == 4 ? 64 : 128, Kin = layer == 2 ? 64 : 128;
            const uint32_t a = layer == 2 ? sA1 : (layer == 3 ? sA2 : sA3);
            const uint32_t b = layer == 2 ? sW2 : (layer == 3 ? sW3 : sW4);
            if (tid == 0)
                mma_chain(tmem + TM_WORK, a, KLBO, 128, 2 * KLBO, false, b, (uint32_t)(Nout / 8) * 128, 128,
                          2 * (uint32_t)(Nout / 8) * 128, false, Nout, Kin, false);
            if (!wait_mma()) break;
            uint8_t* dst = layer == 2 ? A2 : (layer == 3 ? A3 : A4);
            const float* bias = PAR + (layer == 2 ? PB2 : (layer == 3 ? PB3 : PB4));
#pragma unroll 1
            for (int c0 = 16 * h; c0 < Nout; c0 += CS) {
                float z[16], out[16];
                tc::tmem_ld16(tmem + lane_off + TM_WORK + c0, z);
                act16(R, bias, c0, z, out);
                store16(dst, R.r, c0, out);
                if (layer == 4) {
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float2 v = make_float2(out[j], out[j + 1]);
#pragma unroll
                        for (int k = 0; k < 3; ++k) o2[k] = fma2(ld2(PAR + PW5 + 64 * k + c0 + j), v, o2[k]);
                    }
                }
            }
        }
        if (!ok) break;
        float o[3] = {o2[0].x + o2[0].y, o2[1].x + o2[1].y, o2[2].x + o2[2].y};
        // ---- layer 5: the column groups' partial sums (added in group order), the output and
        // the loss (value lanes of group 0), dL/d(outputs) per row into S5
        if (h > 0)
#pragma unroll
            for (int k = 0; k < 3; ++k) X[((h - 1) * 128 + R.r) * 4 + k] = o[k];
        __syncthreads();
        if (h == 0) {
            float ov[3], oxv[3], oyv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int hh = 1; hh < NH; ++hh) o[k] += X[((hh - 1) * 128 + R.r) * 4 + k];
                ov[k] = o[k] + (R.c == 0 ? __ldg(w + OB5 + k) : 0.0f);
                oxv[k] = __shfl_sync(0xffffffffu, o[k], R.lane + 1);
                oyv[k] = __shfl_sync(0xffffffffu, o[k], R.lane + 2);
            }
            float g[3] = {0.0f, 0.0f, 0.0f}, gx[3] = {0.0f, 0.0f, 0.0f}, gy[3] = {0.0f, 0.0f, 0.0f};
            if (valid && R.c == 0) {
                const float t[3] = {t_rho, t_jx / t_rho, t_jy / t_rho};
                const bool iface = t_g > thr;
                const SampleLoss<float> sl = sample_loss<float>(ov, oxv, oyv, t, iface, sx, sy, inv_n, c_phys, c_int, L, hp);
                ld += sl.ld;
                lp += sl.lp;
                li += sl.li;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    g[k] = sl.g[k];
                    gx[k] = sl.gx[k];
                    gy[k] = sl.gy[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float t1 = __shfl_sync(0xffffffffu, gx[k], R.lane - R.c);
                const float t2 = __shfl_sync(0xffffffffu, gy[k], R.lane - R.c);
                S5[R.r * 4 + k] = R.pad ? 0.0f : (R.c == 0 ? g[k] : (R.c == 1 ? t1 : t2));
            }
        }
        __syncthreads();
        const float d5[3] = {S5[R.r * 4], S5[R.r * 4 + 1], S5[R.r * 4 + 2]};
        // ---- layer 5 gradient: warp g < 8 takes features 8 g .. 8 g + 7, lane l the rows l + 32 i
        // (a warp reads 32 consecutive rows of one feature group: no bank conflicts); the 32
        // lanes' partials are folded in lane order (four chains)
        if (warp < 8) {
            float acc[3][8], t8[8];
#pragma unroll
            for (int oo = 0; oo < 3; ++oo)
#pragma unroll
                for (int e = 0; e < 8; ++e) acc[oo][e] = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = R.lane + 32 * i;
                load8(A4, rr, 8 * warp, t8);
#pragma unroll
                for (int oo = 0; oo < 3; ++oo) {
                    const float d = S5[rr * 4 + oo];
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[oo][e] = fmaf(d, t8[e], acc[oo][e]);
                }
            }
#pragma unroll
            for (int oo = 0; oo < 3; ++oo)
#pragma unroll
                for (int e = 0; e < 8; ++e) GP[warp * GP_LD + R.lane * 25 + oo * 8 + e] = acc[oo][e];
        }
        // ---- dL/dA4 and the layer-4 reverse epilogue -> dZ4 (its own buffer: A4 is read by the
        // layer-5 gradient of warps 0-7 at the same time; GP is folded after the next barrier)
#pragma unroll 1
        for (int c0 = 16 * h; c0 < 64; c0 += CS) {
            float dA[16], av[16], own[16], dz[16];
            sample_acts(R, A4, c0, av, own);
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float2 t = fma2(bc2(d5[2]), ld2(PAR + PW5 + 128 + c0 + j),
                                      fma2(bc2(d5[1]), ld2(PAR + PW5 + 64 + c0 + j),
                                           mul2(bc2(d5[0]), ld2(PAR + PW5 + c0 + j))));
                dA[j] = t.x;
                dA[j + 1] = t.y;
            }
            dact16(R, dA, av, own, dz);
            store16(DZ4, R.r, c0, dz);
        }
        // ---- reverse MMAs of layers 4, 3, 2 (with the gradients) and their epilogues
        auto fold5 = [&]() {   // dW5 (GP, in lane order) and db5 (S5) into the slice
            if (tid < 192) {
                const int oo = tid / 64, k = tid % 64;
                const float* g = GP + (k / 8) * GP_LD + oo * 8 + k % 8;
                float a4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int l = 0; l < 32; ++l) a4[l & 3] += g[l * 25];
                acc1(P + OW5 + tid, (a4[0] + a4[1]) + (a4[2] + a4[3]), first);
            } else if (warp >= 8 && warp < 11) {   // db5[o], warp 8 + o: the 40 value rows (lanes 0,
                const int oo = warp - 8;             // 3, ..., 27 of each quadrant), butterfly over lanes
                float a = 0.0f;
                for (int wq = R.lane; wq < 40; wq += 32) a += S5[(32 * (wq / 10) + 3 * (wq % 10)) * 4 + oo];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (R.lane == 0) acc1(P + OB5 + oo, a, first);
            }
        };
#pragma unroll 1
        for (int layer = 4; layer >= 2 && ok; --layer) {
            if (!sync_to_mma()) break;
            const int Nout = layer == 4 ? 64 : 128, Kin = layer == 2 ? 64 : 128;
            const uint32_t dz = layer == 4 ? sDZ4 : (layer == 3 ? sA3 : sA2);   // dZ_l (dZ3, dZ2 over A_l)
            const uint32_t wl = layer == 2 ? sW2 : (layer == 3 ? sW3 : sW4);
            if (tid == 0) {
                if (layer == 4)        // dW4^T += A3^T dZ4
                    mma_rows(tmem + TM_DW4T, sA3, dz, 64, !first);
                else if (layer == 3)   // [dW3 | db3] += dZ3^T [A2 | E2]
                    mma_rows(tmem + TM_DW3, dz, sA2, 144, !first);
                else                   // [db2 | dW2] += dZ2^T [E1 | A1]
                    mma_rows(tmem + TM_DW2, dz, sE1, 80, !first);
                // dA_{l-1} = dZ_l W_l: A = dZ_l K-major (K = out), B = W_l MN-major (K = out, N = in)
                mma_chain(tmem + TM_WORK, dz, KLBO, 128, 2 * KLBO, false, wl, 128, (uint32_t)(Nout / 8) * 128, 256,
                          true, Kin, Nout, false);
            }
            if (layer == 4) fold5();  // CUDA-core work of the previous step, while the MMAs run
            if (!wait_mma()) break;   // all of them: the epilogue overwrites A_{l-1}
            uint8_t* Aact = layer == 2 ? A1 : (layer == 3 ? A2 : A3);
#pragma unroll 1
            for (int c0 = 16 * h; c0 < Kin; c0 += CS) {
                float dA[16], av[16], own[16], dzv[16];
                sample_acts(R, Aact, c0, av, own);   // in flight during the TMEM load
                tc::tmem_ld16(tmem + lane_off + TM_WORK + c0, dA);
                dact16(R, dA, av, own, dzv);
                store16(Aact, R.r, c0, dzv);           // dZ_{l-1} over A_{l-1}
            }
        }
        if (!ok) break;
        // ---- layer-1 and layer-4 bias gradients: [dW1 | db1 ; db4] += [dZ1 | dZ4]^T E1 (A1 and DZ4
        // adjacent), committed here and waited for by the next tile before it rewrites E1 and A1
        if (!sync_to_mma()) break;
        if (tid == 0) {
            mma_rows(tmem + TM_D1, sA1, sE1, 16, !first);
            tc::mma_commit(bar_mma);
        }
        pending = true;
    }
    if (ok && pending) ok = wait_issued();   // the last tile's gradient MMA
    if (ok) {
        // the gradients accumulated in TMEM: rows of [db2 | dW2], [dW3 | db3] and dW4^T; rows < 64
        // of [dW1 | db1], rows >= 64 of db4 (column 2)
        tc::tc_after_sync();
        float v[16];
#pragma unroll 1
        for (int c0 = 16 * h; c0 < 80; c0 += CS) {
            tc::tmem_ld16(tmem + lane_off + TM_DW2 + c0, v);
            if (c0 == 0) {
                P[OB2 + R.r] = v[2];
            } else {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(P + OW2 + R.r * 64 + c0 - 16 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        }
#pragma unroll 1
        for (int c0 = 16 * h; c0 < 144; c0 += CS) {
            tc::tmem_ld16(tmem + lane_off + TM_DW3 + c0, v);
            if (c0 < 128) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(P + OW3 + R.r * 128 + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
                P[OB3 + R.r] = v[2];
            }
        }
#pragma unroll 1
        for (int c0 = 16 * h; c0 < 64; c0 += CS) {
            tc::tmem_ld16(tmem + lane_off + TM_DW4T + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) P[OW4 + (c0 + j) * 128 + R.r] = v[j];
        }
        if (h == 0) {
            tc::tmem_ld16(tmem + lane_off + TM_D1, v);
            if (R.r < 64) {
                P[OW1 + 2 * R.r] = v[0];
                P[OW1 + 2 * R.r + 1] = v[1];
                P[OB1 + R.r] = v[2];
            } else {
                P[OB4 + R.r - 64] = v[2];
            }
        }
    } else {
        // MMAs in flight finish before TMEM is freed (bounded waits, as everywhere): a fresh
        // commit covers every MMA issued; an unobserved earlier commit completes the phase before
        if (tid == 0) {
            atomicOr(err, 1u);
            tc::mma_commit(bar_mma);
        }
        if (pending) {
            (void)tc::mbar_wait(bar_mma, phase);
            phase ^= 1;
        }
        (void)tc::mbar_wait(bar_mma, phase);
    }
    tc::tc_before_sync();
    __syncthreads();
    tc::tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
    double v[3] = {(double)ld, (double)lp, (double)li};
    const int op[3] = {0, 0, 0};
    block_reduce<3>(v, op, reinterpret_cast<double*>(sm + OFF_SC));
    if (tid == 0)
        for (int k = 0; k < 3; ++k) loss_part[blockIdx.x * 4 + k] = ok ? v[k] : NAN;
}

}  // namespace

int train_params_count() { return NPARAM; }
long long train_part_stride() { return PSTRIDE; }

cudaError_t train_grid(int fp64, int* grid) { return fp64 ? grad_setup<double>(grid) : grad_setup<float>(grid); }

template <typename R>
static cudaError_t begin_t(const TrainLat& L, const TrainBufs& b, const float* w32, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.ni, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.err, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    k_train_prep<R><<<UPD_GRID * 4, 256, 0, s>>>(L, w32, static_cast<R*>(b.master), b.ni);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_train_begin(const TrainLat& L, const TrainBufs& b, int fp64, const float* w32, cudaStream_t s) {
    return fp64 ? begin_t<double>(L, b, w32, s) : begin_t<float>(L, b, w32, s);
}

template <typename R>
static cudaError_t epoch_t(const TrainLat& L, const TrainBufs& b, const TrainHyper& hp, long long t, int apply,
                           double* hist_row, cudaStream_t s) {
    int grid = 0;
    cudaError_t e = grad_setup<R>(&grid);
    if (e != cudaSuccess) return e;
    if (grid > b.grid) return cudaErrorInvalidValue;  // partial buffer sized for fewer CTAs
    const long long N = (long long)L.nx * L.ny;
    const long long ntiles = (N + TileOf<R>::T - 1) / TileOf<R>::T;
    k_train_grad<R><<<grid, TR_THREADS, Smem<R>::bytes, s>>>(L, static_cast<const R*>(b.master),
                                                             static_cast<R*>(b.part), b.loss_part, b.ni, hp, ntiles);
    const int nact = (int)(ntiles < grid ? ntiles : grid);
    const double bc1 = apply ? 1.0 / (1.0 - std::pow(hp.beta1, (double)t)) : 1.0;
    const double bc2 = apply ? 1.0 / (1.0 - std::pow(hp.beta2, (double)t)) : 1.0;
    k_train_update<R><<<UPD_GRID, UPD_THREADS, 0, s>>>(static_cast<R*>(b.master), static_cast<R*>(b.m),
                                                       static_cast<R*>(b.v), static_cast<R*>(b.grad),
                                                       static_cast<const R*>(b.part), b.loss_part, b.ni, nact, N, hp,
                                                       bc1, bc2, apply, hist_row);
    note_launches(2);
    return cudaGetLastError();
}

static cudaError_t epoch_tc(const TrainLat& L, const TrainBufs& b, const TrainHyper& hp, long long t, int apply,
                            double* hist_row, cudaStream_t s) {
    static int sms = 0;  // per process (one device)
    if (!sms) {
        cudaError_t e = cudaFuncSetAttribute(k_train_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, ttc::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    if (sms > b.grid) return cudaErrorInvalidValue;
    // BF16 operand image of the weights this epoch starts from
    cudaError_t e = launch_convert_weights_bf16(static_cast<const float*>(b.master), b.wimg, NIN, s);
    if (e != cudaSuccess) return e;
    const long long N = (long long)L.nx * L.ny;
    const long long ntiles = (N + ttc::SPT - 1) / ttc::SPT;
    k_train_grad_tc<<<sms, ttc::THREADS, ttc::SMEM, s>>>(L, static_cast<const float*>(b.master), b.wimg,
                                                        static_cast<float*>(b.part), b.loss_part, b.ni, hp, ntiles, b.err);
    const int nact = (int)(ntiles < sms ? ntiles : sms);
    const double bc1 = apply ? 1.0 / (1.0 - std::pow(hp.beta1, (double)t)) : 1.0;
    const double bc2 = apply ? 1.0 / (1.0 - std::pow(hp.beta2, (double)t)) : 1.0;
    k_train_update<float><<<UPD_GRID, UPD_THREADS, 0, s>>>(static_cast<float*>(b.master), static_cast<float*>(b.m),
                                                           static_cast<float*>(b.v), static_cast<float*>(b.grad),
                                                           static_cast<const float*>(b.part), b.loss_part, b.ni, nact,
                                                           N, hp, bc1, bc2, apply, hist_row);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_train_epoch(const TrainLat& L, const TrainBufs& b, int fp64, const TrainHyper& hp, long long t,
                               int apply, double* hist_row, cudaStream_t s) {
    if (hp.mode == PL_TRAIN_TC) {
        if (fp64) return cudaErrorInvalidValue;
        return epoch_tc(L, b, hp, t, apply, hist_row, s);
    }
    return fp64 ? epoch_t<double>(L, b, hp, t, apply, hist_row, s) : epoch_t<float>(L, b, hp, t, apply, hist_row, s);
}

cudaError_t launch_train_end(const TrainBufs& b, int fp64, float* w32, uint16_t* wbf16, cudaStream_t s) {
    if (fp64) k_train_finish<double><<<UPD_GRID, UPD_THREADS, 0, s>>>(static_cast<const double*>(b.master), w32);
    else k_train_finish<float><<<UPD_GRID, UPD_THREADS, 0, s>>>(static_cast<const float*>(b.master), w32);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_convert_weights_bf16(w32, wbf16, NIN, s);
}

}  // namespace pl
