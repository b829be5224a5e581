// Internal launcher interface between the C ABI (pl_api.cu) and the kernels.
//
// Every kernel of the hot path is table-driven: it reads a device-resident job
// table (one LatDesc per lattice, plus prefix sums of each lattice's work units)
// and loops over virtual work units with a fixed, persistent grid.  A single
// lattice is a table of one; a batch is a table of many.  Because the grids do
// not depend on the table's contents, one captured CUDA graph stays valid while
// the host rewrites the table between replays (jobs admitted and retired).
// Every per-lattice decomposition (reduction blocks, MLP tiles) depends on that
// lattice alone, so each lattice's results are bit-identical alone and in a mix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pinnlbm.h"

namespace pl {

struct DevRecord;

// Kernel-launch accounting (every launcher reports the kernels it enqueued).
void note_launches(long long n);
long long launches_total();

// Geometry of one lattice's arrays inside caller memory (per-lattice kernels:
// initial state and state exchange).
struct LatticeView {
    int nx, ny;
    int storage;
    int pitch;         // elements per stored row (nx rounded up to a multiple of 8)
    long long plane;   // elements per population plane (pitch*ny)
    void* pops[2];     // two-lattice population buffers, 9 planes each
    void* rho;         // scratch (>= 8 nx ny bytes), used as FP64 staging
    DevRecord* rec;
    const pl_droplet* droplets;
};

struct PhysParams {
    double G, tau, rho0, mask_eps, beta_rho, beta_u, threshold;
};

// One lattice of a job table.
struct LatDesc {
    void* pops[2];          // population buffers
    void* rho;              // scratch fields (double for FP64 storage, float otherwise)
    void* jx;
    void* jy;
    void* g;
    void* out3;             // network outputs rho^, u^x, u^y (3 planes of nx*ny)
    double* partials;       // reduction partials, red_blocks x 8
    DevRecord* rec;
    long long plane;        // elements per population plane
    int nx, ny, pitch;
    int phase;              // buffer holding the state when the launch parity is 0
    int nstrips, chunks;    // step decomposition: nstrips x chunks warps
    int red_blocks;         // reduction blocks, a function of nx*ny only
    int has_centre;         // Laplace measurement defined (single droplet)
    unsigned seq0;          // table step count when the lattice joined (its own count = seq - seq0)
    int pad0;
    double G, tau, rho0, mask_eps, beta_rho, beta_u, threshold;
    double cx, cy, width;   // droplet centre and profile width (Laplace)
    int* band;              // the correction's interface band (cells with mask above mask_eps), in cell order
};

struct TabHeader {
    int n;                  // lattices in the table
    int total_blocks;       // sum of red_blocks
    long long total_warps;  // sum of nstrips * chunks
    long long total_tiles;  // sum of ceil(nx*ny / 128)
    int edge_lattices;      // lattices whose FP16 step has strips off the vector path (odd nx,
                            // or ten planes beyond 32-bit element offsets)
    int pad;
};

// Device arrays of a table (capacity cap lattices; prefix arrays have cap+1 entries).
struct TableView {
    const TabHeader* hdr;
    const LatDesc* d;
    const long long* warp_pre;
    const int* blk_pre;
    const long long* tile_pre;
    // Step sequence counter in two slots: a step of parity p reads seq[p] and writes
    // seq[p^1] = seq[p] + 1 (the slot it does not read), so the count advances on the
    // device, also under graph replay.  Feeds the FP16 stochastic-rounding dither.
    unsigned* seq;
};

constexpr int RB_THREADS = 256;         // threads of a reduction block
constexpr int RB_MAX_BLOCKS = 1024;     // reduction blocks per lattice (max)
constexpr int RB_CELLS_PER_THREAD = 32;  // target cells per reduction thread
constexpr int PARTIAL_STRIDE = 8;       // doubles per block partial
constexpr int MLP_TILE = 128;           // cells per network tile
constexpr int STRIP = 60;               // owned columns per step warp

int red_blocks_for(long long cells);
int step_capacity_warps(int storage);   // resident warps of the step kernel on this device

// Per-lattice kernels.
cudaError_t launch_init_droplets(const LatticeView& v, const PhysParams& p, int cur, int n, double rho_in,
                                 double rho_out, double width, double noise_amp, uint64_t seed, cudaStream_t s);
cudaError_t launch_init_from_rho(const LatticeView& v, const PhysParams& p, int cur, const double* d_rho,
                                 cudaStream_t s);
// Convert population plane `plane` of buffer `cur` to (to_f64=1) or from (0) the FP64 array d_buf[nx*ny].
// FP16-offset storage encodes against the buffer's reference plane, which launch_state_ref sets
// from the density of the state first.
cudaError_t launch_state_convert(const LatticeView& v, const PhysParams& p, int cur, double* d_buf, int plane,
                                 int to_f64, cudaStream_t s);
// d_acc = d_buf (first) or d_acc + d_buf (the density of a state uploaded plane by plane).
cudaError_t launch_state_accumulate(const LatticeView& v, double* d_acc, const double* d_buf, int first, cudaStream_t s);
// FP16-offset storage: the reference plane of buffer `cur` from the FP64 density d_rho (no-op otherwise).
cudaError_t launch_state_ref(const LatticeView& v, int cur, const double* d_rho, cudaStream_t s);

// Table kernels (all lattices of a table share `storage`).  FP16-offset storage runs the strips
// off the vector path in a second kernel when `edge` is set (set it when the table may hold
// a lattice with odd nx: always for a batch, whose table changes under a captured graph).
cudaError_t launch_step_tab(const TableView& t, int storage, int parity, cudaStream_t s, bool edge = true);
// Whether a lattice's FP16 step can have strips off the vector path.
__host__ __device__ inline bool f16_edge_lattice(int nx, long long plane) { return (nx & 1) || 10ll * plane > 0xFFFFFFFFll; }
// Metrics of every lattice: moments, Eq. 16 gradient, Eqs. 9-15 sums (+ Laplace where defined).
// moments_current: the moment fields already hold the state's density and momentum (right
// after a correction of the same state, whose apply pass keeps them current), so the moments
// pass is skipped.
cudaError_t launch_metrics_tab(const TableView& t, int storage, int parity, int set_mass0, int laplace,
                               cudaStream_t s, int moments_current = 0);
// Density and momentum fields of every lattice (the network's stencil input reads rho).
cudaError_t launch_moments_tab(const TableView& t, int storage, int parity, cudaStream_t s);
// Network field of every lattice (BF16 tensor cores or SIMT) on n_in = 2 or 11 inputs (11
// reads the density field, which must be current); use_band: the tensor-core form evaluates
// lattices with mask_eps > 0 on their interface band (d.band, rec->band_n) only.  Then the
// correction.
cudaError_t launch_mlp_tab(const TableView& t, int storage, int mlp_mode, int n_in, const float* w32,
                           const uint16_t* wbf16, cudaStream_t s, int use_band = 0);
cudaError_t launch_correction_tab(const TableView& t, int storage, int parity, int mlp_mode, int n_in,
                                  const float* w32, const uint16_t* wbf16, cudaStream_t s);

cudaError_t launch_convert_weights_bf16(const float* w32, uint16_t* wbf16, int n_in, cudaStream_t s);
// Seeded FP32 weight blob (fan-in uniform from SplitMix64, counter = blob index) written on the device.
cudaError_t launch_init_weights(float* w32, int n_in, uint64_t seed, cudaStream_t s);

// Network training (Eqs. 3-8, the 2-input network): the lattice fields it reads (element type
// double for FP64 lattices, float otherwise), its hyper-parameters and its device buffers.
struct TrainLat {
    const void* rho;
    const void* jx;
    const void* jy;
    const void* g;
    int nx, ny;
    double G, rho0, threshold;
};
struct TrainHyper {
    double lr, beta1, beta2, eps, lambda_phys, lambda_int, alpha1, alpha2;
    int mode;                  // PL_TRAIN_SIMT or PL_TRAIN_TC
};
struct TrainBufs {
    void* master;              // weights being trained [train_params_count()]
    void* m;                   // Adam first moments
    void* v;                   // Adam second moments
    void* grad;                // gradient of the last epoch
    void* part;                // per-CTA gradient slices [grid][train_part_stride()]
    double* loss_part;         // per-CTA loss sums [grid][4]
    unsigned long long* ni;    // interface-cell count
    int grid;                  // CTAs the partial buffers hold
    uint16_t* wimg;            // BF16 operand image of the weights (tensor-core mode)
    unsigned* err;             // nonzero: a bounded device wait gave up
};
int train_params_count();
long long train_part_stride();
cudaError_t train_grid(int fp64, int* grid);
// Density, momentum and Eq. 16 gradient fields of every lattice (the training targets).
cudaError_t launch_train_fields_tab(const TableView& t, int storage, int parity, cudaStream_t s);
cudaError_t launch_train_begin(const TrainLat& L, const TrainBufs& b, int fp64, const float* w32, cudaStream_t s);
// One epoch: gradient over all cells, then (apply = 1) the Adam step number t; writes the
// loss terms at the weights the epoch started from to hist_row[4].
cudaError_t launch_train_epoch(const TrainLat& L, const TrainBufs& b, int fp64, const TrainHyper& hp, long long t,
                               int apply, double* hist_row, cudaStream_t s);
// Trained weights -> the FP32 blob and its BF16 image.
cudaError_t launch_train_end(const TrainBufs& b, int fp64, float* w32, uint16_t* wbf16, cudaStream_t s);
cudaError_t launch_selftest_wait(int* d_status, long long limit_ns, cudaStream_t s);
size_t bf16_weight_elems();

}  // namespace pl
