// C ABI of the PINN-LBM hot path, single-lattice calls (declared in include/pinnlbm.h).
//
// Host-side bookkeeping only: argument checks, carving the caller's device buffer,
// the lattice's one-entry job table, stream-ordered launches of the table kernels,
// CUDA-graph capture of the coupled run, and the few synchronising read-backs.  No
// device memory is allocated here: everything lives in the buffer the caller passes in.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "pl_host.h"

namespace pl {

thread_local int g_last_cuda_error = 0;

static std::atomic<long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

int check_params(const pl_params* p) {
    if (!p) return PL_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny >= (1ll << 31)) return PL_ERR_INVALID_ARG;
    if (p->storage != PL_F64 && p->storage != PL_F32 && p->storage != PL_F16_OFFSET) return PL_ERR_INVALID_ARG;
    if (p->storage == PL_F64 && p->mlp != PL_MLP_F64) return PL_ERR_INVALID_ARG;
    if (p->storage != PL_F64 && p->mlp != PL_MLP_F32 && p->mlp != PL_MLP_BF16) return PL_ERR_INVALID_ARG;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return PL_ERR_INVALID_ARG;
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0) || !std::isfinite(p->G)) return PL_ERR_INVALID_ARG;
    if (!(p->mask_eps >= 0.0) || !std::isfinite(p->mask_eps) || !std::isfinite(p->beta_rho) ||
        !std::isfinite(p->beta_u) || !std::isfinite(p->threshold))
        return PL_ERR_INVALID_ARG;
    if (p->mlp_in != 2 && p->mlp_in != 11) return PL_ERR_INVALID_ARG;
    return PL_OK;
}

LatLayout lattice_layout(const pl_params* p) {
    LatLayout L;
    const size_t N = (size_t)p->nx * p->ny;
    L.pitch = row_pitch(p->nx);
    L.plane = (long long)L.pitch * p->ny;
    L.red_blocks = red_blocks_for((long long)N);
    size_t o = 0;
    for (int b = 0; b < 2; ++b) {
        L.pops[b] = o;
        o = align_up(o + (size_t)planes_of(p->storage) * (size_t)L.plane * storage_bytes(p->storage));
    }
    L.scratch = o;  // rho, jx, jy, g, out3[3]: 7 fields (also >= 8N bytes for FP64 staging), then
                    // the correction's band of cell indices (N ints)
    o = align_up(o + 7 * N * scratch_elem_bytes(p->storage) + N * sizeof(int));
    L.partials = o;
    o = align_up(o + (size_t)L.red_blocks * PARTIAL_STRIDE * sizeof(double));
    L.rec = o;
    o = align_up(o + sizeof(DevRecord));
    L.total = o;
    return L;
}

void fill_desc(LatDesc& d, const pl_params* p, const LatLayout& L, char* base) {
    std::memset(&d, 0, sizeof(d));
    const size_t N = (size_t)p->nx * p->ny;
    const size_t se = scratch_elem_bytes(p->storage);
    d.pops[0] = base + L.pops[0];
    d.pops[1] = base + L.pops[1];
    char* sc = base + L.scratch;
    d.rho = sc;
    d.jx = sc + 1 * N * se;
    d.jy = sc + 2 * N * se;
    d.g = sc + 3 * N * se;
    d.out3 = sc + 4 * N * se;
    d.band = reinterpret_cast<int*>(sc + 7 * N * se);
    d.partials = reinterpret_cast<double*>(base + L.partials);
    d.rec = reinterpret_cast<DevRecord*>(base + L.rec);
    d.plane = L.plane;
    d.nx = p->nx;
    d.ny = p->ny;
    d.pitch = L.pitch;
    d.phase = 0;
    d.nstrips = (p->nx + STRIP - 1) / STRIP;
    d.chunks = 1;
    d.red_blocks = L.red_blocks;
    d.has_centre = 0;
    d.G = p->G;
    d.tau = p->tau;
    d.rho0 = p->rho0;
    d.mask_eps = p->mask_eps;
    d.beta_rho = p->beta_rho;
    d.beta_u = p->beta_u;
    d.threshold = p->threshold;
    d.width = 2.0;
}

void set_chunks(LatDesc& d, int rows_per_chunk) {
    if (rows_per_chunk < 1) rows_per_chunk = 1;
    int c = (d.ny + rows_per_chunk - 1) / rows_per_chunk;
    d.chunks = c < 1 ? 1 : c;
}

void set_chunks_single(LatDesc& d, int storage) {
    long long chunks = (long long)step_capacity_warps(storage) / d.nstrips;
    // chunks of at least 8 rows (each chunk walks two rows more than it relaxes), FP64 of at
    // least 2: FP64 lattices are bound by the FP64 rate of the SMs their warps occupy
    const int min_rows = storage == PL_F64 ? 2 : 8;
    const long long max_chunks = d.ny / min_rows > 0 ? d.ny / min_rows : 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    d.chunks = (int)chunks;
}

// Device region of a table: header | descriptors | warp_pre | blk_pre | tile_pre | seq[2].
static size_t tab_off_desc(int cap) { (void)cap; return align_up(sizeof(TabHeader)); }
static size_t tab_off_warp(int cap) { return align_up(tab_off_desc(cap) + (size_t)cap * sizeof(LatDesc)); }
static size_t tab_off_blk(int cap) { return align_up(tab_off_warp(cap) + (size_t)(cap + 1) * sizeof(long long)); }
static size_t tab_off_tile(int cap) { return align_up(tab_off_blk(cap) + (size_t)(cap + 1) * sizeof(int)); }
static size_t tab_off_seq(int cap) { return align_up(tab_off_tile(cap) + (size_t)(cap + 1) * sizeof(long long)); }

size_t Table::bytes(int c) { return align_up(tab_off_seq(c) + 2 * sizeof(unsigned)); }

void Table::carve(char* base, int capacity) {
    cap = capacity;
    dev = base;
    view.hdr = reinterpret_cast<const TabHeader*>(base);
    view.d = reinterpret_cast<const LatDesc*>(base + tab_off_desc(cap));
    view.warp_pre = reinterpret_cast<const long long*>(base + tab_off_warp(cap));
    view.blk_pre = reinterpret_cast<const int*>(base + tab_off_blk(cap));
    view.tile_pre = reinterpret_cast<const long long*>(base + tab_off_tile(cap));
    view.seq = reinterpret_cast<unsigned*>(base + tab_off_seq(cap));
    staging.assign(tab_off_seq(cap), 0);
}

cudaError_t Table::upload(cudaStream_t s) {
    const int n = (int)d.size();
    if (n > cap) return cudaErrorInvalidValue;
    std::memset(staging.data(), 0, staging.size());
    long long* wp = reinterpret_cast<long long*>(staging.data() + tab_off_warp(cap));
    int* bp = reinterpret_cast<int*>(staging.data() + tab_off_blk(cap));
    long long* tp = reinterpret_cast<long long*>(staging.data() + tab_off_tile(cap));
    wp[0] = 0;
    bp[0] = 0;
    tp[0] = 0;
    int edge = 0;
    for (int j = 0; j < n; ++j) {
        const long long N = (long long)d[j].nx * d[j].ny;
        edge += f16_edge_lattice(d[j].nx, d[j].plane) ? 1 : 0;
        wp[j + 1] = wp[j] + (long long)d[j].nstrips * d[j].chunks;
        bp[j + 1] = bp[j] + d[j].red_blocks;
        tp[j + 1] = tp[j] + (N + MLP_TILE - 1) / MLP_TILE;
    }
    TabHeader h{};
    h.n = n;
    h.edge_lattices = edge;
    h.total_warps = wp[n];
    h.total_blocks = bp[n];
    h.total_tiles = tp[n];
    total_warps = wp[n];
    total_blocks = bp[n];
    total_tiles = tp[n];
    edge_lattices = edge;
    std::memcpy(staging.data(), &h, sizeof(h));
    if (n) std::memcpy(staging.data() + tab_off_desc(cap), d.data(), (size_t)n * sizeof(LatDesc));
    return cudaMemcpyAsync(dev, staging.data(), staging.size(), cudaMemcpyHostToDevice, s);
}

cudaError_t Table::reset_seq(cudaStream_t s) { return cudaMemsetAsync(dev + tab_off_seq(cap), 0, 2 * sizeof(unsigned), s); }

}  // namespace pl

using namespace pl;

namespace {

// Lattice buffer: lattice arrays | table (1 entry) | weights FP32 | weights BF16 | droplets.
struct SingleLayout {
    LatLayout lat;
    size_t table, w32, wbf16, droplets, total;
};

SingleLayout single_layout(const pl_params* p) {
    SingleLayout S;
    S.lat = lattice_layout(p);
    size_t o = S.lat.total;
    S.table = o;
    o = align_up(o + Table::bytes(1));
    S.w32 = o;
    o = align_up(o + (size_t)MLP_BLOB_MAX * sizeof(float));
    S.wbf16 = o;
    o = align_up(o + bf16_weight_elems() * sizeof(uint16_t));
    S.droplets = o;
    o = align_up(o + (size_t)PL_MAX_DROPLETS * sizeof(pl_droplet));
    S.total = o;
    return S;
}

struct GraphKey {
    int K, parity;
    bool operator<(const GraphKey& o) const { return K != o.K ? K < o.K : parity < o.parity; }
};
struct GraphEntry {
    cudaGraphExec_t exec;
    long long kernels;  // kernel nodes per replay
};

}  // namespace

struct pl_lattice {
    pl_params p;
    PhysParams phys;
    char* base;
    size_t bytes;
    cudaStream_t stream;
    SingleLayout S;
    LatticeView v;     // per-lattice kernels (init, state exchange)
    Table tab;         // one-entry job table for the table kernels
    float* w32;
    uint16_t* wbf16;
    int cur;           // buffer holding the current post-streaming state
    long long step;
    int initialised;
    int weights_set;
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
    p->mask_eps = 0.0;
    p->beta_rho = 0.1;
    p->beta_u = 0.01;
    p->threshold = 0.01;
    p->mlp_in = 2;
    return PL_OK;
}

int pl_mlp_blob_size(void) { return MLP_BLOB; }

int pl_mlp_blob_size_for(int32_t mlp_in) {
    if (mlp_in != 2 && mlp_in != 11) return PL_ERR_INVALID_ARG;
    return mlp_blob(mlp_in);
}

int pl_lattice_bytes(const pl_params* p, size_t* bytes_out) {
    int st = check_params(p);
    if (st) return st;
    if (!bytes_out) return PL_ERR_INVALID_ARG;
    *bytes_out = single_layout(p).total;
    return PL_OK;
}

int pl_lattice_create(const pl_params* p, void* dev_mem, size_t bytes, void* stream, pl_lattice** out) {
    int st = check_params(p);
    if (st) return st;
    if (!dev_mem || !out || ((uintptr_t)dev_mem % ALIGN) != 0) return PL_ERR_INVALID_ARG;
    SingleLayout S = single_layout(p);
    if (bytes < S.total) return PL_ERR_BUDGET;
    pl_lattice* L = new (std::nothrow) pl_lattice();
    if (!L) return PL_ERR_BUDGET;
    L->p = *p;
    L->phys = PhysParams{p->G, p->tau, p->rho0, p->mask_eps, p->beta_rho, p->beta_u, p->threshold};
    L->base = static_cast<char*>(dev_mem);
    L->bytes = bytes;
    L->stream = static_cast<cudaStream_t>(stream);
    L->S = S;
    LatDesc d;
    fill_desc(d, p, S.lat, L->base);
    set_chunks_single(d, p->storage);
    L->tab.carve(L->base + S.table, 1);
    L->tab.d.assign(1, d);
    LatticeView& v = L->v;
    v.nx = p->nx;
    v.ny = p->ny;
    v.storage = p->storage;
    v.pitch = S.lat.pitch;
    v.plane = S.lat.plane;
    v.pops[0] = d.pops[0];
    v.pops[1] = d.pops[1];
    v.rho = d.rho;
    v.rec = d.rec;
    v.droplets = reinterpret_cast<const pl_droplet*>(L->base + S.droplets);
    L->w32 = reinterpret_cast<float*>(L->base + S.w32);
    L->wbf16 = reinterpret_cast<uint16_t*>(L->base + S.wbf16);
    L->cur = 0;
    L->step = 0;
    L->initialised = 0;
    L->weights_set = 0;
    *out = L;
    return PL_OK;
}

// Table upload + record/counter reset + M0, after a new state has been written to buffer 0.
static int finish_init(pl_lattice* L, int has_centre, double cx, double cy, double width) {
    LatDesc& d = L->tab.d[0];
    d.phase = 0;
    d.has_centre = has_centre;
    d.cx = cx;
    d.cy = cy;
    d.width = width;
    L->cur = 0;
    PL_CUDA(L->tab.upload(L->stream));
    PL_CUDA(L->tab.reset_seq(L->stream));
    PL_CUDA(launch_metrics_tab(L->tab.view, L->p.storage, 0, 1, 0, L->stream));
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
    PL_CUDA(cudaMemsetAsync(L->v.rec, 0, sizeof(DevRecord), L->stream));
    PL_CUDA(launch_init_droplets(L->v, L->phys, 0, n, rho_in, rho_out, width, noise_amp, seed, L->stream));
    int st = finish_init(L, n == 1, n == 1 ? d[0].cx : 0.0, n == 1 ? d[0].cy : 0.0, width);
    if (st) return st;
    L->step = 0;
    L->initialised = 1;
    PL_CUDA(cudaStreamSynchronize(L->stream));  // the host copies may be released now
    return PL_OK;
}

int pl_lattice_init_rho(pl_lattice* L, const double* host_rho) {
    if (!L || !host_rho) return PL_ERR_INVALID_ARG;
    drop_graphs(L);
    const size_t N = (size_t)L->p.nx * L->p.ny;
    double* staging = static_cast<double*>(L->v.rho);  // scratch holds >= 8N bytes
    PL_CUDA(cudaMemsetAsync(L->v.rec, 0, sizeof(DevRecord), L->stream));
    PL_CUDA(cudaMemcpyAsync(staging, host_rho, N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    PL_CUDA(launch_init_from_rho(L->v, L->phys, 0, staging, L->stream));
    int st = finish_init(L, 0, 0.0, 0.0, 2.0);
    if (st) return st;
    PL_CUDA(cudaStreamSynchronize(L->stream));
    L->step = 0;
    L->initialised = 1;
    return PL_OK;
}

int pl_set_mlp_weights(pl_lattice* L, const float* blob, size_t n) {
    if (!L || !blob || n != (size_t)mlp_blob(L->p.mlp_in)) return PL_ERR_INVALID_ARG;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(blob[k])) return PL_ERR_INVALID_ARG;
    L->h_weights.assign(blob, blob + n);
    PL_CUDA(cudaMemcpyAsync(L->w32, L->h_weights.data(), n * sizeof(float), cudaMemcpyHostToDevice, L->stream));
    PL_CUDA(launch_convert_weights_bf16(L->w32, L->wbf16, L->p.mlp_in, L->stream));
    L->weights_set = 1;
    return PL_OK;
}

int pl_init_mlp_weights(pl_lattice* L, uint64_t seed) {
    if (!L) return PL_ERR_INVALID_ARG;
    PL_CUDA(launch_init_weights(L->w32, L->p.mlp_in, seed, L->stream));
    PL_CUDA(launch_convert_weights_bf16(L->w32, L->wbf16, L->p.mlp_in, L->stream));
    L->weights_set = 1;
    return PL_OK;
}

static int do_steps(pl_lattice* L, int n) {
    for (int k = 0; k < n; ++k) {
        PL_CUDA(launch_step_tab(L->tab.view, L->p.storage, L->cur, L->stream, f16_edge_lattice(L->p.nx, L->v.plane)));
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
    PL_CUDA(launch_correction_tab(L->tab.view, L->p.storage, L->cur, L->p.mlp, L->p.mlp_in, L->w32, L->wbf16, L->stream));
    return PL_OK;
}

// Enqueue (or capture) the launches of `nsteps` steps starting at step count `step0`
// and buffer `parity`, with a correction after every step whose count is a multiple of K.
static int enqueue_run(pl_lattice* L, int nsteps, int K, long long step0, int parity) {
    int cur = parity;
    for (int s = 1; s <= nsteps; ++s) {
        PL_CUDA(launch_step_tab(L->tab.view, L->p.storage, cur, L->stream, f16_edge_lattice(L->p.nx, L->v.plane)));
        cur ^= 1;
        if (K > 0 && ((step0 + s) % K) == 0)
            PL_CUDA(launch_correction_tab(L->tab.view, L->p.storage, cur, L->p.mlp, L->p.mlp_in, L->w32, L->wbf16, L->stream));
    }
    return PL_OK;
}

int pl_run(pl_lattice* L, int32_t nsteps, int32_t K) {
    if (!L || nsteps < 0 || K < 0) return PL_ERR_INVALID_ARG;
    if (!L->initialised || (K > 0 && !L->weights_set)) return PL_ERR_STATE;
    if (nsteps == 0) return PL_OK;
    if (K == 0) return do_steps(L, nsteps);
    // Graph unit: one correction interval aligned to multiples of K.  Leading/trailing
    // partial intervals run eagerly.
    int done = 0;
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
    const bool capturable =
        L->stream != nullptr && L->stream != cudaStreamLegacy && L->stream != cudaStreamPerThread;
    if (chunks > 0 && !capturable) {
        int st = enqueue_run(L, chunks * K, K, L->step, L->cur);
        if (st) return st;
        L->cur ^= ((chunks * K) & 1);
        L->step += (long long)chunks * K;
        done += chunks * K;
        chunks = 0;
    }
    for (int c = 0; c < chunks; ++c) {
        GraphKey key{K, L->cur};
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
    const int tail = nsteps - done;
    if (tail > 0) {
        int st = enqueue_run(L, tail, K, L->step, L->cur);
        if (st) return st;
        L->cur ^= (tail & 1);
        L->step += tail;
    }
    return PL_OK;
}

}  // extern "C"

void pl::record_to_metrics(const DevRecord& r, int nx, int ny, int laplace, pl_metric_record* out) {
    const double N = (double)nx * (double)ny;
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
    if (laplace) {
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
    out->status = r.status;
    out->corrections = r.applied;
}

extern "C" {

int pl_metrics(pl_lattice* L, pl_metric_record* out) {
    if (!L || !out) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    const int lap = L->tab.d[0].has_centre;
    PL_CUDA(launch_metrics_tab(L->tab.view, L->p.storage, L->cur, 0, lap, L->stream));
    DevRecord r;
    PL_CUDA(cudaMemcpyAsync(&r, L->v.rec, sizeof(r), cudaMemcpyDeviceToHost, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    record_to_metrics(r, L->p.nx, L->p.ny, lap, out);
    out->step = L->step;
    return PL_OK;
}

int pl_get_rho(pl_lattice* L, double* host_rho) {
    if (!L || !host_rho) return PL_ERR_INVALID_ARG;
    if (!L->initialised) return PL_ERR_STATE;
    const size_t N = (size_t)L->p.nx * L->p.ny;
    PL_CUDA(launch_metrics_tab(L->tab.view, L->p.storage, L->cur, 0, 0, L->stream));
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
    if (!L->weights_set || !L->initialised) return PL_ERR_STATE;
    const size_t N3 = 3 * (size_t)L->p.nx * L->p.ny;
    if (L->p.mlp_in == 11) PL_CUDA(launch_moments_tab(L->tab.view, L->p.storage, L->cur, L->stream));
    PL_CUDA(launch_mlp_tab(L->tab.view, L->p.storage, L->p.mlp, L->p.mlp_in, L->w32, L->wbf16, L->stream));
    const void* out3 = L->tab.d[0].out3;
    if (L->p.storage == PL_F64) {
        PL_CUDA(cudaMemcpyAsync(host_out3, out3, N3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
    } else {
        std::vector<float> tmp(N3);
        PL_CUDA(cudaMemcpyAsync(tmp.data(), out3, N3 * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
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
    const int fresh = !L->initialised;
    if (fresh) PL_CUDA(cudaMemsetAsync(L->v.rec, 0, sizeof(DevRecord), L->stream));
    if (L->p.storage == PL_F16_OFFSET) {
        // the density of the given state (planes summed in order 0..8, FP64) sets the reference
        // plane the populations are then encoded against; the scratch holds both arrays
        double* acc = staging + N;
        for (int i = 0; i < 9; ++i) {
            PL_CUDA(cudaMemcpyAsync(staging, host_f + (size_t)i * N, N * sizeof(double), cudaMemcpyHostToDevice,
                                    L->stream));
            PL_CUDA(launch_state_accumulate(L->v, acc, staging, i == 0, L->stream));
        }
        PL_CUDA(launch_state_ref(L->v, L->cur, acc, L->stream));
    }
    for (int i = 0; i < 9; ++i) {
        PL_CUDA(cudaMemcpyAsync(staging, host_f + (size_t)i * N, N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
        PL_CUDA(launch_state_convert(L->v, L->phys, L->cur, staging, i, 0, L->stream));
    }
    if (fresh) {
        // a state written into buffer cur: make it buffer 0's (phase 0) view consistent
        if (L->cur != 0) return PL_ERR_STATE;
        int st = finish_init(L, 0, 0.0, 0.0, 2.0);
        if (st) return st;
    }
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

int pl_get_mlp_weights(pl_lattice* L, float* host_blob, size_t n) {
    if (!L || !host_blob || n != (size_t)mlp_blob(L->p.mlp_in)) return PL_ERR_INVALID_ARG;
    if (!L->weights_set) return PL_ERR_STATE;
    PL_CUDA(cudaMemcpyAsync(host_blob, L->w32, n * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    return PL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Network training (Eqs. 3-8).  Trainer memory (caller's): master weights, Adam moments and
// the last gradient (4 x blob, element type of the lattice's arithmetic), the per-CTA
// gradient slices of the training kernel, per-CTA loss sums, the loss history and the
// interface-cell count.

struct pl_trainer {
    pl_lattice* lat;
    TrainHyper hp;
    TrainBufs b;
    double* hist;
    int max_epochs;
    int fp64;
    long long t;         // Adam steps taken
    int last_epochs;     // epochs of the last pl_train call
};

namespace {

struct TrainerLayout {
    size_t master, m, v, grad, part, loss_part, hist, ni, err, wimg, total;
    int grid;
};

int trainer_layout(int storage, int max_epochs, TrainerLayout* T) {
    const int fp64 = storage == PL_F64;
    cudaError_t e = train_grid(fp64, &T->grid);
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        (void)cudaGetLastError();
        return PL_ERR_CUDA;
    }
    const size_t es = fp64 ? 8 : 4, P = (size_t)train_params_count();
    size_t o = 0;
    T->master = o; o = align_up(o + P * es);
    T->m = o;      o = align_up(o + P * es);
    T->v = o;      o = align_up(o + P * es);
    T->grad = o;   o = align_up(o + P * es);
    T->part = o;   o = align_up(o + (size_t)T->grid * (size_t)train_part_stride() * es);
    T->loss_part = o; o = align_up(o + (size_t)T->grid * 4 * sizeof(double));
    T->hist = o;   o = align_up(o + (size_t)max_epochs * 4 * sizeof(double));
    T->ni = o;     o = align_up(o + sizeof(unsigned long long));
    T->err = o;    o = align_up(o + sizeof(unsigned));
    T->wimg = o;   o = align_up(o + bf16_weight_elems() * sizeof(uint16_t));
    T->total = o;
    return PL_OK;
}

TrainLat train_lat(pl_lattice* L) {
    const LatDesc& d = L->tab.d[0];
    return TrainLat{d.rho, d.jx, d.jy, d.g, d.nx, d.ny, d.G, d.rho0, d.threshold};
}

bool hyper_ok(const pl_train_params* tp) {
    auto fin = [](double v) { return std::isfinite(v); };
    return tp && (tp->mode == PL_TRAIN_SIMT || tp->mode == PL_TRAIN_TC) && fin(tp->lr) && tp->lr > 0 && fin(tp->beta1) && tp->beta1 >= 0 && tp->beta1 < 1 && fin(tp->beta2) &&
           tp->beta2 >= 0 && tp->beta2 < 1 && fin(tp->eps) && tp->eps > 0 && fin(tp->lambda_phys) &&
           tp->lambda_phys >= 0 && fin(tp->lambda_int) && tp->lambda_int >= 0 && fin(tp->alpha1) && tp->alpha1 >= 0 &&
           fin(tp->alpha2) && tp->alpha2 >= 0;
}

// Targets of the current state, master weights from the blob, interface count.
int train_begin(pl_trainer* T) {
    pl_lattice* L = T->lat;
    PL_CUDA(launch_train_fields_tab(L->tab.view, L->p.storage, L->cur, L->stream));
    PL_CUDA(launch_train_begin(train_lat(L), T->b, T->fp64, L->w32, L->stream));
    return PL_OK;
}

int train_epochs(pl_trainer* T, int epochs) {
    pl_lattice* L = T->lat;
    int st = train_begin(T);
    if (st) return st;
    const TrainLat tl = train_lat(L);
    for (int e = 0; e < epochs; ++e) {
        PL_CUDA(launch_train_epoch(tl, T->b, T->fp64, T->hp, T->t + 1, 1, T->hist + 4 * e, L->stream));
        ++T->t;
    }
    PL_CUDA(launch_train_end(T->b, T->fp64, L->w32, L->wbf16, L->stream));
    T->last_epochs = epochs;
    return PL_OK;
}

}  // namespace

extern "C" {

int pl_train_params_default(pl_train_params* tp) {
    if (!tp) return PL_ERR_INVALID_ARG;
    *tp = pl_train_params{3e-4, 0.9, 0.999, 1e-8, 1.0, 1.0, 1.0, 1.0, PL_TRAIN_SIMT, 0};
    return PL_OK;
}

int pl_trainer_bytes(const pl_params* p, int32_t max_epochs, size_t* bytes_out) {
    int st = check_params(p);
    if (st) return st;
    if (!bytes_out || max_epochs < 1 || p->mlp_in != 2) return PL_ERR_INVALID_ARG;
    TrainerLayout T;
    st = trainer_layout(p->storage, max_epochs, &T);
    if (st) return st;
    *bytes_out = T.total;
    return PL_OK;
}

int pl_trainer_create(pl_lattice* L, const pl_train_params* tp, int32_t max_epochs, void* dev_mem, size_t bytes,
                      pl_trainer** out) {
    if (!L || !out || !dev_mem || ((uintptr_t)dev_mem % ALIGN) != 0 || max_epochs < 1 || !hyper_ok(tp) ||
        L->p.mlp_in != 2 || (tp->mode == PL_TRAIN_TC && L->p.storage == PL_F64))
        return PL_ERR_INVALID_ARG;
    TrainerLayout TL;
    int st = trainer_layout(L->p.storage, max_epochs, &TL);
    if (st) return st;
    if (bytes < TL.total) return PL_ERR_BUDGET;
    pl_trainer* T = new (std::nothrow) pl_trainer();
    if (!T) return PL_ERR_BUDGET;
    char* base = static_cast<char*>(dev_mem);
    T->lat = L;
    T->hp = TrainHyper{tp->lr,          tp->beta1,      tp->beta2,  tp->eps, tp->lambda_phys,
                       tp->lambda_int, tp->alpha1,     tp->alpha2, tp->mode};
    T->b = TrainBufs{base + TL.master,
                     base + TL.m,
                     base + TL.v,
                     base + TL.grad,
                     base + TL.part,
                     reinterpret_cast<double*>(base + TL.loss_part),
                     reinterpret_cast<unsigned long long*>(base + TL.ni),
                     TL.grid,
                     reinterpret_cast<uint16_t*>(base + TL.wimg),
                     reinterpret_cast<unsigned*>(base + TL.err)};
    T->hist = reinterpret_cast<double*>(base + TL.hist);
    T->max_epochs = max_epochs;
    T->fp64 = L->p.storage == PL_F64;
    T->t = 0;
    T->last_epochs = 0;
    const size_t moments = TL.grad - TL.m;  // m and v, adjacent
    cudaError_t e = cudaMemsetAsync(base + TL.m, 0, moments, L->stream);
    if (e != cudaSuccess) {
        delete T;
        g_last_cuda_error = (int)e;
        (void)cudaGetLastError();
        return PL_ERR_CUDA;
    }
    *out = T;
    return PL_OK;
}

int pl_train(pl_trainer* T, int32_t epochs) {
    if (!T || epochs < 1 || epochs > T->max_epochs) return PL_ERR_INVALID_ARG;
    if (!T->lat->initialised || !T->lat->weights_set) return PL_ERR_STATE;
    return train_epochs(T, epochs);
}

int pl_train_losses(pl_trainer* T, double* host_loss, int32_t epochs) {
    if (!T || !host_loss || epochs < 1 || epochs > T->last_epochs) return PL_ERR_INVALID_ARG;
    unsigned err = 0;
    PL_CUDA(cudaMemcpyAsync(host_loss, T->hist, (size_t)epochs * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                            T->lat->stream));
    PL_CUDA(cudaMemcpyAsync(&err, T->b.err, sizeof(unsigned), cudaMemcpyDeviceToHost, T->lat->stream));
    PL_CUDA(cudaStreamSynchronize(T->lat->stream));
    return err ? PL_ERR_TIMEOUT : PL_OK;
}

int pl_train_gradient(pl_trainer* T, double* host_grad, double* host_loss4) {
    if (!T || !host_grad || !host_loss4) return PL_ERR_INVALID_ARG;
    pl_lattice* L = T->lat;
    if (!L->initialised || !L->weights_set) return PL_ERR_STATE;
    int st = train_begin(T);
    if (st) return st;
    PL_CUDA(launch_train_epoch(train_lat(L), T->b, T->fp64, T->hp, 0, 0, T->hist, L->stream));
    const size_t P = (size_t)train_params_count();
    if (T->fp64) {
        PL_CUDA(cudaMemcpyAsync(host_grad, T->b.grad, P * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    } else {
        std::vector<float> tmp(P);
        PL_CUDA(cudaMemcpyAsync(tmp.data(), T->b.grad, P * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
        PL_CUDA(cudaStreamSynchronize(L->stream));
        for (size_t p = 0; p < P; ++p) host_grad[p] = tmp[p];
    }
    PL_CUDA(cudaMemcpyAsync(host_loss4, T->hist, 4 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    PL_CUDA(cudaStreamSynchronize(L->stream));
    T->last_epochs = 0;
    return PL_OK;
}

int pl_run_trained(pl_trainer* T, int32_t nsteps, int32_t K, int32_t epochs) {
    if (!T || nsteps < 0 || K < 1 || epochs < 1 || epochs > T->max_epochs) return PL_ERR_INVALID_ARG;
    pl_lattice* L = T->lat;
    if (!L->initialised || !L->weights_set) return PL_ERR_STATE;
    long long left = nsteps;
    while (left > 0) {
        const long long to_boundary = K - (L->step % K);
        const int n = (int)(left < to_boundary ? left : to_boundary);
        int st = do_steps(L, n);
        if (st) return st;
        left -= n;
        if (L->step % K == 0) {
            st = train_epochs(T, epochs);
            if (st) return st;
            PL_CUDA(launch_correction_tab(L->tab.view, L->p.storage, L->cur, L->p.mlp, L->p.mlp_in, L->w32, L->wbf16,
                                          L->stream));
        }
    }
    return PL_OK;
}

int pl_trainer_destroy(pl_trainer* T) {
    if (!T) return PL_ERR_INVALID_ARG;
    delete T;
    return PL_OK;
}

int pl_selftest_wait_timeout(void* dev_status, int64_t limit_ns, void* stream) {
    if (!dev_status || ((uintptr_t)dev_status % sizeof(int)) || limit_ns < 0 || limit_ns > 5000000000ll)
        return PL_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PL_CUDA(launch_selftest_wait(static_cast<int*>(dev_status), (long long)limit_ns, s));
    int st = 0;
    PL_CUDA(cudaMemcpyAsync(&st, dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PL_CUDA(cudaStreamSynchronize(s));
    return st;
}

}  // extern "C"
