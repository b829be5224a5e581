// C ABI of the PINN-LBM hot path (declared in include/pinnlbm.h).
//
// Host-side bookkeeping only: argument checks, carving the caller's device
// buffer, stream-ordered launches of the kernels, CUDA-graph capture of the
// coupled run, and the few synchronising read-backs.  No device memory is
// allocated here: everything lives in the buffer the caller passes in.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "pinnlbm.h"
#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {
cudaError_t launch_mlp_simt(const LatticeView& v, int mlp_mode, cudaStream_t s);
cudaError_t launch_mlp_tc(const LatticeView& v, cudaStream_t s);

cudaError_t launch_mlp_field(const LatticeView& v, int mlp_mode, cudaStream_t s) {
    if (mlp_mode == PL_MLP_BF16) return launch_mlp_tc(v, s);
    return launch_mlp_simt(v, mlp_mode, s);
}
}  // namespace pl

namespace pl {
static std::atomic<long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace pl

using namespace pl;

static thread_local int g_last_cuda_error = 0;

// On failure: remember the error for pl_last_cuda_error() and clear the
// runtime's last-error slot so that it does not surface in a later call.
#define PL_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            g_last_cuda_error = (int)e_;                      \
            (void)cudaGetLastError();                         \
            return PL_ERR_CUDA;                               \
        }                                                     \
    } while (0)

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

size_t storage_bytes(int storage) { return storage == PL_F64 ? 8 : (storage == PL_F32 ? 4 : 2); }
size_t scratch_elem_bytes(int storage) { return storage == PL_F64 ? 8 : 4; }
// Stored rows are padded to a multiple of 8 populations so that every row, and
// every even column pair, is aligned for vector access.
int row_pitch(int nx) { return (nx + 7) / 8 * 8; }
size_t plane_elems(const pl_params* p) { return (size_t)row_pitch(p->nx) * p->ny; }

constexpr int MLP_BLOB = 64 * 2 + 64 + 128 * 64 + 128 + 128 * 128 + 128 + 64 * 128 + 64 + 3 * 64 + 3;
constexpr int MAX_RED_BLOCKS = 1024;

struct Layout {
    size_t pops[2], scratch, partials, rec, w32, wbf16, droplets, total;
};

int check_params(const pl_params* p) {
    if (!p) return PL_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny >= (1ll << 31)) return PL_ERR_INVALID_ARG;
    if (p->storage != PL_F64 && p->storage != PL_F32 && p->storage != PL_F16_OFFSET) return PL_ERR_INVALID_ARG;
    if (p->storage == PL_F64 && p->mlp != PL_MLP_F64) return PL_ERR_INVALID_ARG;
    if (p->storage != PL_F64 && p->mlp != PL_MLP_F32 && p->mlp != PL_MLP_BF16) return PL_ERR_INVALID_ARG;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return PL_ERR_INVALID_ARG;
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0) || !std::isfinite(p->G)) return PL_ERR_INVALID_ARG;
    if (!std::isfinite(p->rho_ref) || !std::isfinite(p->beta_rho) || !std::isfinite(p->beta_u) ||
        !std::isfinite(p->threshold))
        return PL_ERR_INVALID_ARG;
    return PL_OK;
}

Layout layout_for(const pl_params* p) {
    Layout L;
    const size_t N = (size_t)p->nx * p->ny;
    size_t o = 0;
    for (int b = 0; b < 2; ++b) {
        L.pops[b] = o;
        o = align_up(o + 9 * plane_elems(p) * storage_bytes(p->storage));
    }
    L.scratch = o;  // rho, jx, jy, g, out3[3]: 7 fields (also >= 8N bytes for FP64 staging)
    o = align_up(o + 7 * N * scratch_elem_bytes(p->storage));
    L.partials = o;
    o = align_up(o + (size_t)MAX_RED_BLOCKS * 8 * sizeof(double));
    L.rec = o;
    o = align_up(o + sizeof(DevRecord));
    L.w32 = o;
    o = align_up(o + (size_t)MLP_BLOB * sizeof(float));
    L.wbf16 = o;
    o = align_up(o + bf16_weight_elems() * sizeof(uint16_t));
    L.droplets = o;
    o = align_up(o + (size_t)PL_MAX_DROPLETS * sizeof(pl_droplet));
    L.total = o;
    return L;
}

}  // namespace

struct GraphKey {
    int K, parity, nsteps;
    bool operator<(const GraphKey& o) const {
        if (K != o.K) return K < o.K;
        if (parity != o.parity) return parity < o.parity;
        return nsteps < o.nsteps;
    }
};

struct GraphEntry {
    cudaGraphExec_t exec;
    long long kernels;  // kernel nodes per replay
};

struct pl_lattice {
    pl_params p;
    PhysParams phys;
    char* base;
    size_t bytes;
    cudaStream_t stream;
    LatticeView v;
    StepTiling tiling;
    int cur;                 // buffer holding the current post-streaming state
    long long step;
    int initialised;
    int weights_set;
    int has_centre;
    double cx0, cy0, width;
    std::vector<pl_droplet> h_droplets;
    std::vector<float> h_weights;
    std::map<GraphKey, GraphEntry> graphs;
};

static void drop_graphs(pl_lattice* L) {
    for (auto& kv : L->graphs) cudaGraphExecDestroy(kv.second.exec);
    L->graphs.clear();
}

extern "C" {

const char* pl_status_string(int s) {
    switch (s) {
        case PL_OK: return "ok";
        case PL_ERR_INVALID_ARG: return "invalid argument";
        case PL_ERR_CUDA: return "CUDA error";
        case PL_ERR_BUDGET: return "insufficient memory or budget";
        case PL_ERR_NONPHYSICAL: return "correction rejected: non-physical state";
        case PL_ERR_TIMEOUT: return "device wait timed out";
        case PL_ERR_STATE: return "invalid call for the current state";
    }
    return "unknown status";
}

int pl_last_cuda_error(void) { return g_last_cuda_error; }

int pl_kernel_launches(int64_t* out) {
    if (!out) return PL_ERR_INVALID_ARG;
    *out = launches_total();
    return PL_OK;
}

int pl_params_default(pl_params* p, int32_t nx, int32_t ny) {
    if (!p) return PL_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->storage = PL_F32;
    p->mlp = PL_MLP_BF16;
    p->G = -5.5;
    p->tau = 1.0;
    p->rho0 = 1.0;
    p->rho_ref = 1.075;
    p->beta_rho = 0.1;
    p->beta_u = 0.01;
    p->threshold = 0.01;
    return PL_OK;
}

int pl_mlp_blob_size(void) { return MLP_BLOB; }

int pl_lattice_bytes(const pl_params* p, size_t* bytes_out) {
    int st = check_params(p);
    if (st) return st;
    if (!bytes_out) return PL_ERR_INVALID_ARG;
    *bytes_out = layout_for(p).total;
    return PL_OK;
}

int pl_lattice_create(const pl_params* p, void* dev_mem, size_t bytes, void* stream, pl_lattice** out) {
    int st = check_params(p);
    if (st) return st;
    if (!dev_mem || !out || ((uintptr_t)dev_mem % ALIGN) != 0) return PL_ERR_INVALID_ARG;
    Layout Ly = layout_for(p);
    if (bytes < Ly.total) return PL_ERR_BUDGET;
    pl_lattice* L = new (std::nothrow) pl_lattice();
    if (!L) return PL_ERR_BUDGET;
    L->p = *p;
    L->phys = PhysParams{p->G, p->tau, p->rho0, p->rho_ref, p->beta_rho, p->beta_u, p->threshold};
    L->base = static_cast<char*>(dev_mem);
    L->bytes = bytes;
    L->stream = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)p->nx * p->ny;
    const size_t se = scratch_elem_bytes(p->storage);
    LatticeView& v = L->v;
    v.nx = p->nx;
    v.ny = p->ny;
    v.storage = p->storage;
    v.pitch = row_pitch(p->nx);
    v.plane = (long long)plane_elems(p);
    v.pops[0] = L->base + Ly.pops[0];
    v.pops[1] = L->base + Ly.pops[1];
    char* sc = L->base + Ly.scratch;
    v.rho = sc;
    v.jx = sc + 1 * N * se;
    v.jy = sc + 2 * N * se;
    v.g = sc + 3 * N * se;
    v.out3 = sc + 4 * N * se;
    v.partials = reinterpret_cast<double*>(L->base + Ly.partials);
    v.max_blocks = MAX_RED_BLOCKS;
    v.rec = reinterpret_cast<DevRecord*>(L->base + Ly.rec);
    v.w32 = reinterpret_cast<const float*>(L->base + Ly.w32);
    v.wbf16 = reinterpret_cast<const uint16_t*>(L->base + Ly.wbf16);
    v.droplets = reinterpret_cast<const pl_droplet*>(L->base + Ly.droplets);
    L->tiling = default_tiling(p->nx, p->ny);
    L->cur = 0;
    L->step = 0;
    L->initialised = 0;
    L->weights_set = 0;
    L->has_centre = 0;
    *out = L;
    return PL_OK;
}

static int reset_record(pl_lattice* L) {
    PL_CUDA(cudaMemsetAsync(L->v.rec, 0, sizeof(DevRecord), L->stream));
    return PL_OK;
}

int pl_lattice_init_droplets(pl_lattice* L, const pl_droplet* d, int n, double rho_in, double rho_out, double width,
                             double noise_amp, uint64_t seed) {
    if (!L || n < 0 || n > PL_MAX_DROPLETS || (n > 0 && !d)) return PL_ERR_INVALID_ARG;
    if (!std::isfinite(rho_in) || !std::isfinite(rho_out) || !(width > 0.0) || !std::isfinite(noise_amp))
        return PL_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(d[k].cx) || !std::isfinite(d[k].cy) || !(d[k].r >= 0.0)) return PL_ERR_INVALID_ARG;
    drop_graphs(L);
    L->h_droplets.assign(d, d + n);
    if (n > 0)
        PL_CUDA(cudaMemcpyAsync(const_cast<pl_droplet*>(L->v.droplets), L->h_droplets.data(), n * sizeof(pl_droplet),
                                cudaMemcpyHostToDevice, L->stream));
    int st = reset_record(L);
    if (st) return st;
    L->cur = 0;
    PL_CUDA(launch_init_droplets(L->v, L->phys, L->cur, n, rho_in, rho_out, width, noise_amp, seed, L->stream));
    PL_CUDA(launch_metrics(L->v, L->phys, L->cur, 0, 0.0, 0.0, width, 1, L->stream));
    L->step = 0;
    L->initialised = 1;
    L->has_centre = n == 1;  // the Laplace measurement is defined for a single droplet
    L->cx0 = n > 0 ? d[0].cx : 0.0;
    L->cy0 = n > 0 ? d[0].cy : 0.0;
    L->width = width;
    // keep the host copy alive until the copy has been consumed
    PL_CUDA(cudaStreamSynchronize(L->stream));
    return PL_OK;
}

int pl_lattice_init_rho(pl_lattice* L, const double* host_rho) {
    if (!L || !host_rho) return PL_ERR_INVALID_ARG;
    drop_graphs(L);
    const size_t N = (size_t)L->p.nx * L->p.ny;
    double* staging = static_cast<double*>(L->v.rho);  // scratch holds >= 8N bytes
    int st = reset_record(L);
    if (st) return st;
    L->cur = 0;
    PL_CUDA(cudaMemcpyAsync(staging, host_rho, N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    PL_CUDA(launch_init_from_rho(L->v, L->phys, L->cur, staging, L->stream));
    PL_CUDA(launch_metrics(L->v, L->phys, L->cur, 0, 0.0, 0.0, 2.0, 1, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    L->step = 0;
    L->initialised = 1;
    L->has_centre = 0;
    return PL_OK;
}

int pl_set_mlp_weights(pl_lattice* L, const float* blob, size_t n) {
    if (!L || !blob || n != (size_t)MLP_BLOB) return PL_ERR_INVALID_ARG;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(blob[k])) return PL_ERR_INVALID_ARG;
    L->h_weights.assign(blob, blob + n);
    PL_CUDA(cudaMemcpyAsync(const_cast<float*>(L->v.w32), L->h_weights.data(), n * sizeof(float),
                            cudaMemcpyHostToDevice, L->stream));
    PL_CUDA(launch_convert_weights_bf16(L->v.w32, const_cast<uint16_t*>(L->v.wbf16), L->stream));
    L->weights_set = 1;
    return PL_OK;
}

static int do_steps(pl_lattice* L, int n) {
    for (int k = 0; k < n; ++k) {
        PL_CUDA(launch_step(L->v, L->phys, L->cur, L->tiling, L->stream));
        L->cur ^= 1;
    }
    L->step += n;
    return PL_OK;
}

int pl_step(pl_lattice* L, int32_t n) {
    if (!L || n < 0) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    return do_steps(L, n);
}

int pl_apply_correction(pl_lattice* L) {
    if (!L) return PL_ERR_INVALID_ARG;
    if (!L->initialised || !L->weights_set) return PL_ERR_STATE;
    PL_CUDA(launch_correction(L->v, L->phys, L->cur, L->p.mlp, L->stream));
    return PL_OK;
}

// Enqueue (or capture) the launches of `nsteps` steps starting at step count
// `step0`, with a correction after every step whose count is a multiple of K.
static int enqueue_run(pl_lattice* L, int nsteps, int K, long long step0, int parity) {
    int cur = parity;
    for (int s = 1; s <= nsteps; ++s) {
        PL_CUDA(launch_step(L->v, L->phys, cur, L->tiling, L->stream));
        cur ^= 1;
        if (K > 0 && ((step0 + s) % K) == 0) PL_CUDA(launch_correction(L->v, L->phys, cur, L->p.mlp, L->stream));
    }
    return PL_OK;
}

int pl_run(pl_lattice* L, int32_t nsteps, int32_t K) {
    if (!L || nsteps < 0 || K < 0) return PL_ERR_INVALID_ARG;
    if (!L->initialised || (K > 0 && !L->weights_set)) return PL_ERR_STATE;
    if (nsteps == 0) return PL_OK;
    // Graph unit: one correction interval aligned to multiples of K (or 1 step
    // without corrections).  Leading/trailing partial intervals run eagerly.
    int done = 0;
    if (K > 0) {
        int lead = (int)((K - (L->step % K)) % K);
        if (lead > nsteps) lead = nsteps;
        if (lead > 0) {
            int st = enqueue_run(L, lead, K, L->step, L->cur);
            if (st) return st;
            L->cur ^= (lead & 1);
            L->step += lead;
            done = lead;
        }
        int chunks = (nsteps - done) / K;
        // The legacy default stream cannot be captured: enqueue eagerly there.
        const bool capturable = L->stream != nullptr && L->stream != cudaStreamLegacy &&
                                L->stream != cudaStreamPerThread;
        if (chunks > 0 && !capturable) {
            int st = enqueue_run(L, chunks * K, K, L->step, L->cur);
            if (st) return st;
            L->cur ^= ((chunks * K) & 1);
            L->step += (long long)chunks * K;
            done += chunks * K;
            chunks = 0;
        }
        if (chunks > 0) {
            for (int c = 0; c < chunks; ++c) {
                GraphKey key{K, L->cur, K};
                auto it = L->graphs.find(key);
                if (it == L->graphs.end()) {
                    cudaGraph_t g;
                    PL_CUDA(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
                    const long long before = launches_total();
                    int st = enqueue_run(L, K, K, 0, L->cur);
                    const long long captured = launches_total() - before;
                    note_launches(-captured);  // captured, not executed: counted at each replay
                    cudaError_t ce = cudaStreamEndCapture(L->stream, &g);
                    if (st) return st;
                    PL_CUDA(ce);
                    cudaGraphExec_t ge;
                    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
                    cudaGraphDestroy(g);
                    PL_CUDA(ie);
                    it = L->graphs.emplace(key, GraphEntry{ge, captured}).first;
                }
                PL_CUDA(cudaGraphLaunch(it->second.exec, L->stream));
                note_launches(it->second.kernels);
                L->cur ^= (K & 1);
                L->step += K;
            }
            done += chunks * K;
        }
        int tail = nsteps - done;
        if (tail > 0) {
            int st = enqueue_run(L, tail, K, L->step, L->cur);
            if (st) return st;
            L->cur ^= (tail & 1);
            L->step += tail;
        }
        return PL_OK;
    }
    return do_steps(L, nsteps);
}

int pl_metrics(pl_lattice* L, pl_metric_record* out) {
    if (!L || !out) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    PL_CUDA(launch_metrics(L->v, L->phys, L->cur, L->has_centre, L->cx0, L->cy0, L->width, 0, L->stream));
    DevRecord r;
    PL_CUDA(cudaMemcpyAsync(&r, L->v.rec, sizeof(r), cudaMemcpyDeviceToHost, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    const double N = (double)L->p.nx * (double)L->p.ny;
    std::memset(out, 0, sizeof(*out));
    out->mass = r.mass;
    out->count = r.count;
    out->W = (double)r.count / N;
    out->G_max = r.gmax;
    out->delta_rho = r.rho_max - r.rho_min;
    out->W_eff = r.gmax > 0.0 ? r.sum_g / (r.gmax * N) : 0.0;
    out->E_int = r.sum_g2;
    out->rho_max = r.rho_max;
    out->rho_min = r.rho_min;
    out->sum_g = r.sum_g;
    out->sum_g2 = r.sum_g2;
    if (L->has_centre) {
        out->R_eq = r.R_eq;
        out->rho_in = r.rho_in;
        out->rho_out = r.rho_out;
        out->p_in = r.p_in;
        out->p_out = r.p_out;
        out->dP = r.p_in - r.p_out;
    } else {
        out->R_eq = out->rho_in = out->rho_out = out->p_in = out->p_out = out->dP = NAN;
    }
    out->mass0 = r.mass0;
    out->step = L->step;
    out->status = r.status;
    out->corrections = r.applied;
    return PL_OK;
}

int pl_get_rho(pl_lattice* L, double* host_rho) {
    if (!L || !host_rho) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    const size_t N = (size_t)L->p.nx * L->p.ny;
    PL_CUDA(launch_metrics(L->v, L->phys, L->cur, 0, 0.0, 0.0, 2.0, 0, L->stream));
    if (L->p.storage == PL_F64) {
        PL_CUDA(cudaMemcpyAsync(host_rho, L->v.rho, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
    } else {
        std::vector<float> tmp(N);
        PL_CUDA(cudaMemcpyAsync(tmp.data(), L->v.rho, N * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
        for (size_t c = 0; c < N; ++c) host_rho[c] = tmp[c];
    }
    return PL_OK;
}

int pl_get_mlp_field(pl_lattice* L, double* host_out3) {
    if (!L || !host_out3) return PL_ERR_INVALID_ARG;
    if (!L->weights_set) return PL_ERR_STATE;
    const size_t N3 = 3 * (size_t)L->p.nx * L->p.ny;
    PL_CUDA(launch_mlp_field(L->v, L->p.mlp, L->stream));
    if (L->p.storage == PL_F64) {
        PL_CUDA(cudaMemcpyAsync(host_out3, L->v.out3, N3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
    } else {
        std::vector<float> tmp(N3);
        PL_CUDA(cudaMemcpyAsync(tmp.data(), L->v.out3, N3 * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
        for (size_t c = 0; c < N3; ++c) host_out3[c] = tmp[c];
    }
    return PL_OK;
}

int pl_get_state(pl_lattice* L, double* host_f, int64_t* step) {
    if (!L || !host_f) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    const size_t N = (size_t)L->p.nx * L->p.ny;
    double* staging = static_cast<double*>(L->v.rho);
    for (int i = 0; i < 9; ++i) {
        PL_CUDA(launch_state_convert(L->v, L->phys, L->cur, staging, i, 1, L->stream));
        PL_CUDA(cudaMemcpyAsync(host_f + (size_t)i * N, staging, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    }
    PL_CUDA(cudaStreamSynchronize(L->stream));
    if (step) *step = L->step;
    return PL_OK;
}

int pl_set_state(pl_lattice* L, const double* host_f, int64_t step) {
    if (!L || !host_f || step < 0) return PL_ERR_INVALID_ARG;
    const size_t N = (size_t)L->p.nx * L->p.ny;
    for (size_t k = 0; k < 9 * N; ++k)
        if (!std::isfinite(host_f[k])) return PL_ERR_INVALID_ARG;
    drop_graphs(L);
    double* staging = static_cast<double*>(L->v.rho);
    if (!L->initialised) {
        int st = reset_record(L);
        if (st) return st;
    }
    for (int i = 0; i < 9; ++i) {
        PL_CUDA(cudaMemcpyAsync(staging, host_f + (size_t)i * N, N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
        PL_CUDA(launch_state_convert(L->v, L->phys, L->cur, staging, i, 0, L->stream));
    }
    if (!L->initialised) PL_CUDA(launch_metrics(L->v, L->phys, L->cur, 0, 0.0, 0.0, 2.0, 1, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    L->step = step;
    L->initialised = 1;
    return PL_OK;
}

int pl_lattice_status(pl_lattice* L) {
    if (!L) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_OK;
    int s = 0;
    PL_CUDA(cudaMemcpyAsync(&s, &L->v.rec->status, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    return s;
}

int pl_destroy(pl_lattice* L) {
    if (!L) return PL_ERR_INVALID_ARG;
    drop_graphs(L);
    delete L;
    return PL_OK;
}

}  // extern "C"
