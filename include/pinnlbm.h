/*
 * pinnlbm.h - C ABI of the GB300 (sm_103a) PINN-LBM droplet hot path.
 *
 * Method: arXiv 2504.10539, "Physics-Informed Neural Networks for Enhanced
 * Interface Preservation in Lattice Boltzmann Multiphase Simulations".
 *   - lattice update: Sec. II-A, Eq. 1 (D2Q9 pseudopotential lattice,
 *     psi = rho0 (1 - exp(-rho/rho0)), Shan-Chen force, force-shifted
 *     equilibrium, BGK collision, periodic streaming);
 *   - network N(x, y) -> (rho, u_x, u_y): Sec. II-B Eq. 2, architecture Sec. III-B;
 *   - coupling / correction: Sec. II-C (a correction weighted toward the
 *     interface regions, applied every few steps rather than every step);
 *   - metrics: Sec. II-D Eqs. 9-13, discretised in Sec. IV-E Eqs. 14-16;
 *   - droplet set-up: Sec. III-A.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: PL_OK (0) or a negative PL_ERR_*.
 *     No C++ exception crosses this boundary.  A call that fails with
 *     PL_ERR_INVALID_ARG or PL_ERR_STATE has changed nothing.
 *   - The CALLER owns all device memory.  pl_lattice_bytes() says how many
 *     bytes a lattice needs; the caller allocates them (e.g. a torch uint8
 *     tensor on the GPU) and passes the pointer to pl_lattice_create(), which
 *     carves it up and never allocates device memory itself.  The pointer must
 *     be 256-byte aligned and stay valid until pl_destroy().
 *   - The CALLER owns the stream (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream).  All work is enqueued on it asynchronously,
 *     except the calls documented as synchronising (pl_metrics, pl_get_*,
 *     pl_lattice_status), which wait for that stream.
 *   - Host pointers passed in are only read during the call; the library keeps
 *     its own copies where it needs the data later.
 *   - The library owns the opaque handle (host memory), freed by pl_destroy().
 *   - Population exchange format (pl_get_state / pl_set_state): FP64, layout
 *     f[i][y][x] (i = 0..8 direction-major, x fastest), with the D2Q9 order
 *     c_0=(0,0), c_1..4=(1,0),(0,1),(-1,0),(0,-1), c_5..8=(1,1),(-1,1),(-1,-1),(1,-1).
 */
#ifndef PINNLBM_H
#define PINNLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PL_API __attribute__((visibility("default")))
#else
#define PL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PL_OK 0
#define PL_ERR_INVALID_ARG (-1) /* bad pointer, size, enum or value                 */
#define PL_ERR_CUDA (-2)        /* a CUDA runtime call failed; see pl_last_cuda_error */
#define PL_ERR_BUDGET (-3)      /* not enough caller memory / device budget           */
#define PL_ERR_NONPHYSICAL (-4) /* correction would give rho <= 0 or non-finite state */
#define PL_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                 */
#define PL_ERR_STATE (-6)       /* call not valid in the handle's current state       */

/* Population storage (bytes per population: 8, 4, 2). */
#define PL_F64 0        /* FP64 storage, FP64 arithmetic                          */
#define PL_F32 1        /* FP32 storage, FP32 arithmetic                          */
#define PL_F16_OFFSET 2 /* FP16 offsets from each population's source reference,  */
                        /* FP32 arithmetic (see below)                           */

/* FP16-offset storage (PL_F16_OFFSET; the paper fixes no number format).  A population
 * buffer holds ten FP16 planes: the offsets h_0..h_8 and the reference densities r.  The
 * population f_i at cell x is stored relative to the reference density of the cell it
 * streamed from, scaled by 2^10,
 *     f_i(x) = 2^-10 h_i(x) + Wr_i * r(x - c_i),  Wr = (1824, 456, 456, 456, 456, 114, 114, 114, 114) / 4096
 * (Wr = (4104/4096) w, proportional to the lattice weights w; Wr_i * r is exact in FP32).  A
 * time step writes r(x) = fp16(rho(x)) with the populations cell x pushes, so each offset is
 * the population's departure from its source cell's rest equilibrium; the rest population
 * of each cell takes the cell's mass balance, and every offset is rounded stochastically
 * (unbiased).  Bytes per cell update: 2 x (9 + 1) x 2 = 40. */

/* Network arithmetic for the correction. */
#define PL_MLP_F64 0  /* FP64 on CUDA cores                                        */
#define PL_MLP_F32 1  /* FP32 on CUDA cores                                        */
#define PL_MLP_BF16 2 /* BF16 operands on tcgen05 tensor cores, FP32 accumulation  */

#define PL_MAX_DROPLETS 4096

/* Lattice parameters.  G, tau, rho0: Sec. II-A / Sec. III-A (the paper's g and tau);
 * beta_rho, beta_u: gains of the interface correction; threshold: the |grad rho| threshold
 * of the interface width W (Eq. 9; the paper uses 0.01); mask_eps: the correction's
 * interface band (Sec. II-C weights the correction toward the interface, Sec. IV-D samples
 * the interface adaptively; the band is this library's reading): cells whose mask
 * m = |grad rho| / max |grad rho| is not above mask_eps count as outside the interface (m = 0:
 * not corrected, not in the projections, no network evaluation).  mask_eps = 0 (default) is
 * the full correction; 0 < mask_eps evaluates the network on the band only. */
typedef struct pl_params {
    int32_t nx, ny;   /* lattice size, each >= 1, nx*ny < 2^31                  */
    int32_t storage;  /* PL_F64 / PL_F32 / PL_F16_OFFSET                        */
    int32_t mlp;      /* PL_MLP_*                                               */
    double G;         /* interaction strength (< 0 attracts); the paper: -5.5   */
    double tau;       /* BGK relaxation time, > 0.5; the paper: 1.0             */
    double rho0;      /* pseudopotential scale, > 0                             */
    double mask_eps;  /* interface band of the correction, >= 0 (default 0)     */
    double beta_rho;  /* correction gain on density  (default 0.1)              */
    double beta_u;    /* correction gain on momentum (default 0.01)             */
    double threshold; /* Eq. 9 gradient threshold    (default 0.01)             */
    int32_t mlp_in;   /* network inputs: 2 = the paper's cell centre (x^, y^)    */
                      /* (default); 11 = (x^, y^) and the density of the cell   */
                      /* and its 8 neighbours in velocity order c_0..c_8        */
                      /* (a stencil variant the paper does not have)            */
    int32_t reserved; /* 0                                                      */
} pl_params;

/* One droplet of the initial state: centre (cx, cy) in lattice units, radius r. */
typedef struct pl_droplet {
    double cx, cy, r;
} pl_droplet;

/* Metric record (FP64).  Eqs. 9-15 plus the mass and the Laplace measurement
 * about the droplet's centre (NaN unless the lattice was initialised from
 * exactly one droplet). */
typedef struct pl_metric_record {
    double mass;      /* sum of rho over the lattice                         */
    double W;         /* Eq. 9:  fraction of cells with |grad rho| > threshold */
    double G_max;     /* Eq. 10: max |grad rho|                               */
    double delta_rho; /* Eq. 11: rho_max - rho_min                            */
    double W_eff;     /* Eq. 12/14: sum|grad rho| / (G_max * N); 0 if G_max=0 */
    double E_int;     /* Eq. 13/15: sum |grad rho|^2 (dx = dy = 1)            */
    double rho_max, rho_min, sum_g, sum_g2;
    int64_t count;    /* cells with |grad rho| > threshold                    */
    double R_eq, rho_in, rho_out, p_in, p_out, dP; /* Laplace measurement      */
    double mass0;     /* reference mass M0 of the correction's projection     */
    int64_t step;     /* time steps taken since initialisation                */
    int32_t status;   /* PL_OK, or the lattice's sticky error (e.g. NONPHYSICAL) */
    int32_t corrections; /* corrections applied so far                        */
} pl_metric_record;

typedef struct pl_lattice pl_lattice;

/* Status text (static string, never NULL). */
PL_API const char* pl_status_string(int status);
/* cudaError_t value of the most recent failing CUDA call in this thread (0 if none). */
PL_API int pl_last_cuda_error(void);
/* Number of CUDA kernels this library has launched in this process (a graph
 * replay counts each of its kernel nodes), for launch accounting. */
PL_API int pl_kernel_launches(int64_t* out);
/* Fill p with the defaults: storage F32, mlp BF16, G=-5.5, tau=1, rho0=1, mask_eps=0,
 * beta_rho=0.1, beta_u=0.01, threshold=0.01, size nx x ny. */
PL_API int pl_params_default(pl_params* p, int32_t nx, int32_t ny);

/* Bytes of caller device memory one lattice with these parameters needs. */
PL_API int pl_lattice_bytes(const pl_params* p, size_t* bytes_out);

/* Create a lattice over caller memory dev_mem[0, bytes) (>= pl_lattice_bytes,
 * 256-byte aligned) that enqueues on `stream`.  No device work is done. */
PL_API int pl_lattice_create(const pl_params* p, void* dev_mem, size_t bytes, void* stream, pl_lattice** out);

/* Initial state (Sec. III-A): rho = rho_out + (rho_in - rho_out) * max_k 1/2 (1 - tanh((d_k - r_k)/width))
 * + noise_amp * (2 U - 1), d_k the periodic minimum-image distance from cell (x, y)
 * to droplet k, U = SplitMix64 uniform of output index y*nx + x for `seed`;
 * u = 0, f_i = w_i rho.  n in [0, PL_MAX_DROPLETS].  Resets the step count, the
 * correction count and the status, and records M0 = mass of the stored state. */
PL_API int pl_lattice_init_droplets(pl_lattice* lat, const pl_droplet* droplets, int n, double rho_in,
                             double rho_out, double width, double noise_amp, uint64_t seed);

/* Initial state from a host density field rho[y][x] (FP64, nx*ny values): f_i = w_i rho. */
PL_API int pl_lattice_init_rho(pl_lattice* lat, const double* host_rho);

/* Network weights (Sec. III-B, 2 -> 64 -> 128 -> 128 -> 64 -> 3, tanh hidden, linear output):
 * FP32 blob W1[64x2] b1[64] W2[128x64] b2[128] W3[128x128] b3[128] W4[64x128] b4[64] W5[3x64] b5[3],
 * row-major W[out][in]; n must equal pl_mlp_blob_size_for(params.mlp_in).  Copied to the device
 * (and converted to the tensor-core operand layout) on the lattice's stream. */
PL_API int pl_mlp_blob_size(void);
/* Blob length for a network with mlp_in inputs (2 or 11; W1 is 64 x mlp_in), or
 * PL_ERR_INVALID_ARG for another input count. */
PL_API int pl_mlp_blob_size_for(int32_t mlp_in);
PL_API int pl_set_mlp_weights(pl_lattice* lat, const float* host_blob, size_t n);
/* Seeded weights for the network of Sec. III-B (the configurations' "seed-initialised"
 * network; the paper fixes no distribution, so the fan-in uniform is used): entry k of the
 * blob above, in blob order, is (2 U - 1) / sqrt(fan_in) with U = top 53 bits of SplitMix64
 * output k for `seed` (the generator of pl_lattice_init_droplets) divided by 2^53 and fan_in
 * the input width of the entry's layer (params.mlp_in for layer 1), rounded to FP32.
 * Written on the device on the lattice's stream (no host data); replaces any earlier
 * weights.  Read them back with pl_get_mlp_weights. */
PL_API int pl_init_mlp_weights(pl_lattice* lat, uint64_t seed);

/* n >= 0 time steps of Eq. 1 on the device (no host synchronisation). */
PL_API int pl_step(pl_lattice* lat, int32_t n);

/* One interface correction (Sec. II-C step 3), all on the device:
 *   g = |grad rho| (Eq. 16), m = g / max g, (rho^, u^) = N(x^, y^) at the cell
 *   centre mapped to [-1, 1]; drho = beta_rho m (rho^ - rho) projected so that
 *   the total mass returns to M0; dj = beta_u m (rho' u^ - j) projected to keep
 *   the total momentum; f_i += f_i^eq(rho', u') - f_i^eq(rho, u) where m > 0.
 * If any corrected density would be <= 0 or non-finite, the state is left
 * unchanged and the lattice's status becomes PL_ERR_NONPHYSICAL (read it with
 * pl_lattice_status or pl_metrics).  Requires weights (PL_ERR_STATE otherwise). */
PL_API int pl_apply_correction(pl_lattice* lat);

/* Coupled run (Sec. II-C): nsteps time steps; after every step whose count
 * (since initialisation) is a multiple of K (K > 0) a correction is applied.
 * K = 0 runs pure LBM.  The step/correction sequence is captured once in a
 * CUDA graph per (K, buffer parity) and replayed. */
PL_API int pl_run(pl_lattice* lat, int32_t nsteps, int32_t K);

/* Metrics of the current state (Eqs. 9-16, mass, Laplace).  Synchronises the stream. */
PL_API int pl_metrics(pl_lattice* lat, pl_metric_record* out);

/* Density field rho[y][x] (FP64, nx*ny values) of the current state.  Synchronises. */
PL_API int pl_get_rho(pl_lattice* lat, double* host_rho);

/* Network field N(x^, y^) at every cell centre (the tensor used by the correction):
 * host_out3[3][ny][nx] = (rho^, u^_x, u^_y), FP64.  Requires weights.  Synchronises. */
PL_API int pl_get_mlp_field(pl_lattice* lat, double* host_out3);

/* Checkpoint: the current populations in the exchange format (9*nx*ny FP64) and
 * the step count.  pl_get_state synchronises; pl_set_state encodes into the
 * lattice's storage type (rounding to nearest for F32; for FP16-offset storage the
 * references r = fp16(rho) with rho summed over i = 0..8 in order in FP64, then
 * h_i = fp16(2^10 (f_i - Wr_i r(x - c_i))) computed in FP64) and sets the step count. */
PL_API int pl_get_state(pl_lattice* lat, double* host_f, int64_t* step);
PL_API int pl_set_state(pl_lattice* lat, const double* host_f, int64_t step);

/* Allocation-free metrics (the paper has no counterpart).  Some callers cannot allocate
 * device memory: code running inside an allocator or a memory-pool callback (where a
 * cudaMalloc would re-enter the allocator), or a host that must not grow its device
 * footprint after start-up.  They cannot hand the library the scratch buffer that
 * pl_lattice_create carves up, so this call keeps its scratch in a static device array.
 * It fills the record fields mass, W, G_max, delta_rho, W_eff, E_int, rho_max, rho_min,
 * sum_g, sum_g2 and count (threshold: the gradient threshold that W and count use), the
 * same quantities pl_metrics returns, of populations that the caller passes at dev_pops
 * (device memory, element type given by `storage`, 9 planes of ny rows of `pitch` >= nx
 * elements, x fastest; FP16-offset storage: 10 planes, the offsets h_0..h_8 and the reference
 * densities, as described at PL_F16_OFFSET; rho_ref is unused).  The Laplace fields
 * and mass0 are NaN, step, status and corrections 0.  The record is written to host memory
 * at `out`.  Its scratch (density field, block partials, record) is a static device array
 * of 8.07 MB that every GPU loading the library keeps until the process exits; the call
 * makes no cudaMalloc, cudaFree or allocating library call.  Lattices above 1,048,576
 * cells are rejected with PL_ERR_BUDGET (and a message on stderr).  Every call looks up the
 * array's address on the calling thread's current device, which must be the device that
 * holds dev_pops.  All calls share the one array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  Enqueues on `stream` and synchronises it. */
PL_API int pl_metrics_noalloc(const void* dev_pops, int32_t nx, int32_t ny, int32_t pitch, int32_t storage,
                              double rho_ref, double threshold, void* stream, pl_metric_record* out);

/* Sticky lattice status (PL_OK or the first device-detected error).  Synchronises. */
PL_API int pl_lattice_status(pl_lattice* lat);

/* Free the handle; the caller's device memory is not touched. */
PL_API int pl_destroy(pl_lattice* lat);

/* Network weights currently on the device (the FP32 blob, n = pl_mlp_blob_size_for(
 * params.mlp_in)); after pl_train these are the trained weights.  Synchronises. */
PL_API int pl_get_mlp_weights(pl_lattice* lat, float* host_blob, size_t n);

/* ---------------------------------------------------------------------------------
 * Network training on the lattice state (Sec. II-C step 2; loss Eqs. 3-8; Sec. III-B:
 * learning rate 3e-4, 300 epochs per coupling step), for the paper's 2-input network
 * (params.mlp_in = 2).  The paper leaves the following open; the library's reading:
 *   - samples: every cell, input (x^, y^) as for the correction; one epoch = one
 *     gradient step on the loss over all cells;
 *   - targets: rho = sum f_i and u = j / rho of the state when pl_train is called;
 *   - L_data (Eq. 4): mean over the cells of |N - (rho, u_x, u_y)|^2;
 *   - L_phys (Eqs. 5-7): mean over the cells of r_c^2 + |r_m|^2, r_c = div(rho u),
 *     r_m = div(rho u u) + grad p, on the network's fields and their spatial derivatives
 *     (lattice units, d/dx = (2/nx) d/dx^); no time derivative (N has no time input),
 *     p = rho/3 + G psi^2/6, stress taken as zero;
 *   - L_int (Eq. 8): mean over the cells with |grad rho| (Eq. 16) above params.threshold
 *     of -alpha1 q + alpha2 q^2, q = |grad rho_N|^2 (the signs the text describes);
 *   - optimizer: Adam with bias correction, no weight decay; its moments and step count
 *     live in the trainer and persist across pl_train calls;
 *   - between calls the network is the lattice's FP32 blob (the correction's weights):
 *     each call starts from it and writes the trained weights back to it (and to the
 *     tensor-core operand image).
 * Arithmetic: FP64 for FP64 lattices, FP32 otherwise (CUDA cores).
 * --------------------------------------------------------------------------------- */
/* Training arithmetic (pl_train_params.mode). */
#define PL_TRAIN_SIMT 0 /* CUDA cores: FP64 for FP64 lattices, FP32 otherwise (default)        */
#define PL_TRAIN_TC 1   /* tcgen05 tensor cores for layers 2-4 (forward, reverse, weight
                           gradient) and for the bias and layer-1 gradients: BF16 operands,
                           FP32 accumulation; the layer-1 forward pass, layer 5, the loss and
                           the tanh terms in FP32; FP32 and FP16-offset lattices only          */

typedef struct pl_train_params {
    double lr;          /* Adam step size (default 3e-4, Sec. III-B)          */
    double beta1;       /* Adam first-moment decay (0.9)                      */
    double beta2;       /* Adam second-moment decay (0.999)                   */
    double eps;         /* Adam denominator guard (1e-8)                      */
    double lambda_phys; /* Eq. 3 weight of L_phys (1)                         */
    double lambda_int;  /* Eq. 3 weight of L_int (1)                          */
    double alpha1;      /* Eq. 8 weight of q = |grad rho_N|^2 (1)             */
    double alpha2;      /* Eq. 8 weight of q^2 (1)                            */
    int32_t mode;       /* PL_TRAIN_SIMT (default) or PL_TRAIN_TC             */
    int32_t reserved;   /* 0                                                  */
} pl_train_params;

typedef struct pl_trainer pl_trainer;

PL_API int pl_train_params_default(pl_train_params* tp);
/* Bytes of caller device memory a trainer for lattices of this storage type needs with a
 * loss history of max_epochs >= 1 entries (depends on the current device's SM count). */
PL_API int pl_trainer_bytes(const pl_params* p, int32_t max_epochs, size_t* bytes_out);
/* Trainer of lattice `lat` over caller memory dev_mem[0, bytes) (256-byte aligned, valid
 * until pl_trainer_destroy); enqueues on the lattice's stream.  Adam's moments start at
 * zero.  PL_ERR_INVALID_ARG for a lattice with mlp_in != 2, invalid hyper-parameters
 * (lr > 0, 0 <= beta < 1, eps > 0, lambdas and alphas finite and >= 0) or PL_TRAIN_TC on an
 * FP64 lattice. */
PL_API int pl_trainer_create(pl_lattice* lat, const pl_train_params* tp, int32_t max_epochs, void* dev_mem,
                             size_t bytes, pl_trainer** out);
/* epochs (1..max_epochs) training epochs on the lattice's current state; the loss
 * history of the call is kept for pl_train_losses.  Requires weights and a state
 * (PL_ERR_STATE otherwise).  No host synchronisation. */
PL_API int pl_train(pl_trainer* tr, int32_t epochs);
/* Loss history of the last pl_train call, host_loss[epochs][4] = (L, L_data, L_phys,
 * L_int), each evaluated at the weights its epoch started from.  Synchronises.  Returns
 * PL_ERR_TIMEOUT if a bounded device wait of the tensor-core kernel gave up during the call
 * (the losses of the affected epochs are NaN). */
PL_API int pl_train_losses(pl_trainer* tr, double* host_loss, int32_t epochs);
/* The gradient of Eq. 3 with respect to the blob (host_grad[pl_mlp_blob_size()], FP64)
 * and the loss terms (host_loss4[4] as above) at the lattice's current weights and state;
 * nothing is updated.  Synchronises. */
PL_API int pl_train_gradient(pl_trainer* tr, double* host_grad, double* host_loss4);
/* Coupled run with training (Sec. II-C): nsteps time steps; after every step whose count
 * is a multiple of K (K > 0), `epochs` training epochs on the state, then one correction
 * with the trained network. */
PL_API int pl_run_trained(pl_trainer* tr, int32_t nsteps, int32_t K, int32_t epochs);
/* Free the handle; the caller's device memory is not touched.  A trainer refers to its
 * lattice: destroy it before the lattice (pl_destroy). */
PL_API int pl_trainer_destroy(pl_trainer* tr);

/* Self-test of the device-side failure detection: one thread waits, with the bounded
 * mbarrier wait used by the tensor-core kernel, on a barrier that nothing arrives on;
 * after limit_ns (<= 5 s) the wait gives up and the kernel writes PL_ERR_TIMEOUT to the
 * caller's device int at dev_status.  Returns that status (PL_ERR_TIMEOUT when the
 * detection works).  Synchronises `stream`. */
PL_API int pl_selftest_wait_timeout(void* dev_status, int64_t limit_ns, void* stream);

/* ---------------------------------------------------------------------------------
 * Batched and served lattices (many independent droplet-relaxation jobs of different
 * sizes advancing together; Sec. II-C's coupling loop applied to every job).
 *
 * A batch owns one caller buffer: a fixed head (pl_batch_overhead_bytes) and an arena
 * from which each admitted job's lattice memory (pl_batch_job_bytes) is carved.  The
 * buffer size is the device-memory budget: a job that does not fit is refused with
 * PL_ERR_BUDGET and may be resubmitted after others retire.  All jobs of a batch share
 * the storage type, the network arithmetic, the network weights and the correction
 * interval K.  The batch advances in intervals of K steps; each interval runs, for every
 * active job, K time steps, one interface correction and the metrics, as one replayed
 * CUDA graph whose kernels read the device-resident job table.  A job's step count is
 * rounded up to a multiple of K; it retires at the end of the interval that reaches it.
 * Each job's results are bit-identical whether it runs alone or with others.
 * --------------------------------------------------------------------------------- */
typedef struct pl_batch pl_batch;

/* Result of a retired job: its id, steps taken, size, status and final metrics. */
typedef struct pl_job_result {
    int64_t id;
    int64_t steps;
    int32_t nx, ny;
    int32_t status;   /* PL_OK or the job's sticky error (e.g. PL_ERR_NONPHYSICAL) */
    int32_t pad;
    pl_metric_record metrics;
} pl_job_result;

/* Bytes of the fixed head of a batch holding up to max_jobs jobs (weights, job table,
 * droplet staging); the rest of the caller buffer is the arena. */
PL_API int pl_batch_overhead_bytes(int32_t max_jobs, size_t* bytes_out);
/* Arena bytes one job with these parameters takes. */
PL_API int pl_batch_job_bytes(const pl_params* p, size_t* bytes_out);
/* Create a batch over caller memory dev_mem[0, bytes) (256-byte aligned) on `stream`. */
PL_API int pl_batch_create(int32_t storage, int32_t mlp, int32_t K, int32_t max_jobs, void* dev_mem, size_t bytes,
                           void* stream, pl_batch** out);
/* Network weights shared by all jobs (layout of pl_set_mlp_weights). */
PL_API int pl_batch_set_mlp_weights(pl_batch* b, const float* host_blob, size_t n);
/* Seeded weights shared by all jobs, as pl_init_mlp_weights, for a network with mlp_in (2
 * or 11) inputs; PL_ERR_INVALID_ARG if the batch already holds a network of another input
 * count. */
PL_API int pl_batch_init_mlp_weights(pl_batch* b, int32_t mlp_in, uint64_t seed);
/* Admit one job: lattice parameters (storage must match the batch), initial droplets
 * (as pl_lattice_init_droplets) and the number of steps.  PL_ERR_BUDGET if its memory or
 * a job slot is not available now.  Writes the job id. */
PL_API int pl_batch_submit(pl_batch* b, const pl_params* p, const pl_droplet* droplets, int n, double rho_in,
                           double rho_out, double width, double noise_amp, uint64_t seed, int64_t steps,
                           int64_t* job_id);
/* Advance every active job by `intervals` intervals of K steps (asynchronous). */
PL_API int pl_batch_advance(pl_batch* b, int32_t intervals);
/* Collect up to max results of retired jobs, oldest first.  Synchronises the stream. */
PL_API int pl_batch_poll(pl_batch* b, pl_job_result* out, int32_t max, int32_t* n_out);
/* Active jobs, their total cells, and arena use. */
PL_API int pl_batch_info(pl_batch* b, int32_t* active, int64_t* cells, size_t* arena_used, size_t* arena_total);
/* Populations of an active job in the exchange format, and its step count.  Synchronises. */
PL_API int pl_batch_get_state(pl_batch* b, int64_t job_id, double* host_f, int64_t* steps);
/* Choose the step kernel's decomposition (rows per warp chunk) for the current job mix by
 * timing candidates (cached per storage and total-cells octave; force = 1 re-times). */
PL_API int pl_batch_autotune(pl_batch* b, int32_t force, int32_t* rows_per_chunk);
/* Latest metric records (as of the last completed interval) of up to max active jobs, in
 * admission order.  Synchronises the stream. */
PL_API int pl_batch_metrics(pl_batch* b, pl_job_result* out, int32_t max, int32_t* n_out);
/* Device time of the last interval: its K step launches and the whole interval (steps,
 * correction, metrics), from events recorded inside the interval.  Synchronises. */
PL_API int pl_batch_interval_times(pl_batch* b, float* steps_ms, float* interval_ms);
/* Free the handle; the caller's device memory is not touched. */
PL_API int pl_batch_destroy(pl_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* PINNLBM_H */
