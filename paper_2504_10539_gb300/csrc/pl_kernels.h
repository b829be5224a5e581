// Internal launcher interface between the C ABI (pl_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pinnlbm.h"

namespace pl {

struct DevRecord;

// Kernel-launch accounting (every launcher reports the kernels it enqueued).
void note_launches(long long n);
long long launches_total();

// Geometry of one lattice's arrays inside caller memory.
struct LatticeView {
    int nx, ny;
    int storage;
    int pitch;         // elements per stored row (nx rounded up to a multiple of 8)
    long long plane;   // elements per population plane (pitch*ny)
    void* pops[2];     // two-lattice population buffers, 9 planes each
    // scratch fields, element type = double for F64 storage, float otherwise
    void* rho;
    void* jx;
    void* jy;
    void* g;
    void* out3;        // network outputs rho^, u^_x, u^_y (3 planes)
    double* partials;  // per-block reduction partials
    int max_blocks;    // capacity of partials (blocks)
    DevRecord* rec;
    const float* w32;        // FP32 weight blob (device)
    const uint16_t* wbf16;   // BF16 tensor-core operand copy of W2..W4 (device)
    const pl_droplet* droplets;
};

struct PhysParams {
    double G, tau, rho0, rho_ref, beta_rho, beta_u, threshold;
};

// Step kernel tiling: TX threads per CTA (TX-2 owned columns), TY rows per CTA.
struct StepTiling {
    int tx, ty;
};
StepTiling default_tiling(int nx, int ny);

cudaError_t launch_init_droplets(const LatticeView& v, const PhysParams& p, int cur, int n, double rho_in,
                                 double rho_out, double width, double noise_amp, uint64_t seed, cudaStream_t s);
cudaError_t launch_init_from_rho(const LatticeView& v, const PhysParams& p, int cur, const double* d_rho,
                                 cudaStream_t s);
cudaError_t launch_step(const LatticeView& v, const PhysParams& p, int src, StepTiling t, cudaStream_t s);
// Convert population plane `plane` of buffer `cur` to (to_f64=1) or from (0) the FP64 array d_buf[nx*ny].
cudaError_t launch_state_convert(const LatticeView& v, const PhysParams& p, int cur, double* d_buf, int plane,
                                 int to_f64, cudaStream_t s);

// Metrics: moments + gradient reductions (+ Laplace when has_centre).
cudaError_t launch_metrics(const LatticeView& v, const PhysParams& p, int cur, int has_centre, double cx,
                           double cy, double width, int set_mass0, cudaStream_t s);
int reduction_blocks(const LatticeView& v);

// Correction: network field + 3 reduction phases + apply.
cudaError_t launch_correction(const LatticeView& v, const PhysParams& p, int cur, int mlp_mode, cudaStream_t s);
cudaError_t launch_mlp_field(const LatticeView& v, int mlp_mode, cudaStream_t s);
cudaError_t launch_convert_weights_bf16(const float* w32, uint16_t* wbf16, cudaStream_t s);
size_t bf16_weight_elems();

}  // namespace pl
