// C ABI of batched and served lattices (declared in include/pinnlbm.h).
//
// A batch owns one caller buffer: a fixed head (weights, job table, droplet staging)
// and an arena from which each admitted job's lattice memory is carved (first-fit,
// coalescing free list).  Admission fails with PL_ERR_BUDGET when the arena or the
// job table is full; the caller retries after jobs retire, so requests that arrive
// while others run are admitted as memory and slots free up (continuous batching).
//
// The batch advances in coupling intervals of K steps.  One interval is a captured
// CUDA graph: K launches of the step kernel over every lattice of the job table, the
// interface correction of every lattice, and the metrics of every lattice.  The
// kernels use fixed persistent grids and read the device-resident table, so the same
// graph is replayed while the host rewrites the table between intervals (admissions,
// retirements, re-tuned step decomposition).  Jobs end at an interval boundary: the
// step count of a job is rounded up to a multiple of K.
//
// The step decomposition (rows per warp chunk) is chosen by an autotuner that times
// candidate decompositions with repeated launches of one step parity (each rereads the
// same source buffer and rewrites the same destination, so trials change no state) and
// caches the winner per (storage, total-cells octave).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "pl_host.h"

using namespace pl;

namespace {

// First-fit allocator over [0, size) in 256-byte units; free blocks are coalesced.
class Arena {
   public:
    void reset(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    // Returns the offset, or SIZE_MAX if no free block is large enough.
    size_t alloc(size_t bytes) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

   private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Job {
    int64_t id;
    pl_params p;
    LatLayout L;
    size_t off;
    int64_t target, done;
    LatDesc desc;
};

struct GraphEntry {
    cudaGraphExec_t exec;
    long long kernels;
};

// Batch head: weights FP32 | weights BF16 | table | droplet staging.
struct Head {
    size_t w32, wbf16, table, drops, total;
};
Head head_layout(int max_jobs) {
    Head h;
    size_t o = 0;
    h.w32 = o;
    o = align_up(o + (size_t)MLP_BLOB_MAX * sizeof(float));
    h.wbf16 = o;
    o = align_up(o + bf16_weight_elems() * sizeof(uint16_t));
    h.table = o;
    o = align_up(o + Table::bytes(max_jobs));
    h.drops = o;
    o = align_up(o + (size_t)PL_MAX_DROPLETS * sizeof(pl_droplet));
    h.total = o;
    return h;
}

constexpr int TUNE_CANDIDATES[] = {8, 16, 24, 32, 48, 64, 96, 128};

}  // namespace

struct pl_batch {
    int storage, mlp, K, max_jobs;
    char* base;
    size_t bytes;
    cudaStream_t stream;
    Head H;
    Table tab;
    Arena arena;
    char* arena_base;
    std::vector<Job> jobs;      // active jobs, in table order
    int64_t next_id;
    int parity;                 // steps taken by the batch, mod 2
    unsigned steps_total;       // steps taken by the batch (the device step counter's value)
    int weights_set;
    int table_dirty;
    int mass0_pending;
    int rows_per_chunk;
    std::map<std::pair<int, int>, int> tune_cache;
    std::map<int, GraphEntry> graphs;   // by parity at the start of an interval | 2 if edge lattices
    // results of retired jobs: device records copied into pinned host slots
    DevRecord* h_records;       // pinned, max_jobs slots
    std::vector<int> free_slots;
    struct Pending {
        pl_job_result r;
        int slot;
        int laplace;
    };
    std::vector<Pending> pending;
    int mlp_in;                 // network inputs of every job (0 until weights or a job fix it)
    float* h_weights;           // pinned staging of the FP32 weight blob
    cudaEvent_t ev_w;           // its last upload (the buffer is rewritten only after it)
    std::vector<pl_droplet> h_drops;
    cudaEvent_t ev[3];          // interval start, end of the K steps, end of the interval
    DevRecord* h_live;          // pinned, max_jobs slots (pl_batch_metrics)
};

static void drop_graphs(pl_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

static void rebuild_table(pl_batch* b) {
    b->tab.d.clear();
    for (auto& j : b->jobs) {
        set_chunks(j.desc, b->rows_per_chunk);
        b->tab.d.push_back(j.desc);
    }
    b->table_dirty = 1;
}

static int upload_table(pl_batch* b) {
    if (!b->table_dirty) return PL_OK;
    PL_CUDA(b->tab.upload(b->stream));
    b->table_dirty = 0;
    return PL_OK;
}

static long long total_cells(const pl_batch* b) {
    long long c = 0;
    for (auto& j : b->jobs) c += (long long)j.p.nx * j.p.ny;
    return c;
}

static int octave(long long v) {
    int k = 0;
    while (v > 1) {
        v >>= 1;
        ++k;
    }
    return k;
}

// Time each candidate decomposition with repeated step launches of one parity.
static int autotune(pl_batch* b, int force) {
    if (b->jobs.empty()) return PL_OK;
    const std::pair<int, int> key{b->storage, octave(total_cells(b))};
    auto it = b->tune_cache.find(key);
    if (it != b->tune_cache.end() && !force) {
        if (b->rows_per_chunk != it->second) {
            b->rows_per_chunk = it->second;
            rebuild_table(b);
        }
        return upload_table(b);
    }
    cudaEvent_t e0, e1;
    PL_CUDA(cudaEventCreate(&e0));
    PL_CUDA(cudaEventCreate(&e1));
    // Every trial launch reads the same buffer and writes the other (same parity): the state
    // is unchanged.  The device is warmed up first (clocks ramp up under load), then every
    // candidate is timed in two passes of opposite order, keeping its best time, so that no
    // candidate profits from running later than the others.
    const int nc = (int)(sizeof(TUNE_CANDIDATES) / sizeof(TUNE_CANDIDATES[0]));
    float t_best[sizeof(TUNE_CANDIDATES) / sizeof(TUNE_CANDIDATES[0])];
    for (int c = 0; c < nc; ++c) t_best[c] = 1e30f;
    // the device table must list the current jobs before any trial launch: after retirements
    // and admissions the one on the device still names retired jobs, whose arena space may
    // already hold a new job's state (a trial step would write over it)
    {
        const int st = upload_table(b);
        if (st) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
    }
    const bool edge = b->tab.edge_lattices > 0;
    for (int k = 0; k < 20; ++k) PL_CUDA(launch_step_tab(b->tab.view, b->storage, b->parity, b->stream, edge));
    for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < nc; ++q) {
            const int c = pass == 0 ? q : nc - 1 - q;
            b->rows_per_chunk = TUNE_CANDIDATES[c];
            rebuild_table(b);
            int st = upload_table(b);
            if (st) return st;
            const bool ed = b->tab.edge_lattices > 0;
            PL_CUDA(launch_step_tab(b->tab.view, b->storage, b->parity, b->stream, ed));  // warm-up
            PL_CUDA(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < 3; ++k) PL_CUDA(launch_step_tab(b->tab.view, b->storage, b->parity, b->stream, ed));
            PL_CUDA(cudaEventRecord(e1, b->stream));
            PL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            PL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < t_best[c]) t_best[c] = ms;
        }
    }
    int best_r = TUNE_CANDIDATES[0];
    float best = 1e30f;
    for (int c = 0; c < nc; ++c)
        if (t_best[c] < best) {
            best = t_best[c];
            best_r = TUNE_CANDIDATES[c];
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->rows_per_chunk = best_r;
    b->tune_cache[key] = best_r;
    rebuild_table(b);
    return upload_table(b);
}

// One interval: K steps, correction, metrics.  Events around the K step launches (graph
// event-record nodes when captured) time the step kernels of every interval.  The FP16
// edge-path step kernel is launched only while some lattice of the table needs it (a graph
// is captured for each case).
static int enqueue_interval(pl_batch* b, int parity, bool captured) {
    int cur = parity;
    const bool edge = b->tab.edge_lattices > 0;
    const unsigned flags = captured ? cudaEventRecordExternal : cudaEventRecordDefault;
    PL_CUDA(cudaEventRecordWithFlags(b->ev[0], b->stream, flags));
    for (int s = 0; s < b->K; ++s) {
        PL_CUDA(launch_step_tab(b->tab.view, b->storage, cur, b->stream, edge));
        cur ^= 1;
    }
    PL_CUDA(cudaEventRecordWithFlags(b->ev[1], b->stream, flags));
    PL_CUDA(launch_correction_tab(b->tab.view, b->storage, cur, b->mlp, b->mlp_in,
                                  reinterpret_cast<const float*>(b->base + b->H.w32),
                                  reinterpret_cast<const uint16_t*>(b->base + b->H.wbf16), b->stream));
    PL_CUDA(launch_metrics_tab(b->tab.view, b->storage, cur, 0, 1, b->stream, 1));  // moments kept by the apply pass
    PL_CUDA(cudaEventRecordWithFlags(b->ev[2], b->stream, flags));
    return PL_OK;
}

extern "C" {

PL_API int pl_batch_overhead_bytes(int32_t max_jobs, size_t* bytes_out) {
    if (max_jobs < 1 || max_jobs > (1 << 20) || !bytes_out) return PL_ERR_INVALID_ARG;
    *bytes_out = head_layout(max_jobs).total;
    return PL_OK;
}

PL_API int pl_batch_job_bytes(const pl_params* p, size_t* bytes_out) {
    int st = check_params(p);
    if (st) return st;
    if (!bytes_out) return PL_ERR_INVALID_ARG;
    *bytes_out = lattice_layout(p).total;
    return PL_OK;
}

PL_API int pl_batch_create(int32_t storage, int32_t mlp, int32_t K, int32_t max_jobs, void* dev_mem, size_t bytes,
                           void* stream, pl_batch** out) {
    if (!out || !dev_mem || ((uintptr_t)dev_mem % ALIGN) != 0 || K < 1 || max_jobs < 1 || max_jobs > (1 << 20))
        return PL_ERR_INVALID_ARG;
    if (storage != PL_F64 && storage != PL_F32 && storage != PL_F16_OFFSET) return PL_ERR_INVALID_ARG;
    if (storage == PL_F64 ? mlp != PL_MLP_F64 : (mlp != PL_MLP_F32 && mlp != PL_MLP_BF16)) return PL_ERR_INVALID_ARG;
    const Head H = head_layout(max_jobs);
    if (bytes < H.total) return PL_ERR_BUDGET;
    pl_batch* b = new (std::nothrow) pl_batch();
    if (!b) return PL_ERR_BUDGET;
    b->storage = storage;
    b->mlp = mlp;
    b->K = K;
    b->max_jobs = max_jobs;
    b->base = static_cast<char*>(dev_mem);
    b->bytes = bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    b->H = H;
    b->tab.carve(b->base + H.table, max_jobs);
    b->arena_base = b->base + H.total;
    b->arena.reset(bytes - H.total);
    b->next_id = 1;
    b->parity = 0;
    b->steps_total = 0;
    b->weights_set = 0;
    b->table_dirty = 1;
    b->mass0_pending = 0;
    b->rows_per_chunk = 32;
    b->h_records = nullptr;
    b->h_live = nullptr;
    b->h_weights = nullptr;
    b->ev_w = nullptr;
    b->mlp_in = 0;
    b->ev[0] = b->ev[1] = b->ev[2] = nullptr;
    // pinned host slots for records and the weight upload (host allocations; no device
    // memory is allocated)
    cudaError_t e = cudaMallocHost(&b->h_records, sizeof(DevRecord) * (size_t)max_jobs);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_live, sizeof(DevRecord) * (size_t)max_jobs);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_weights, sizeof(float) * (size_t)MLP_BLOB_MAX);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_w, cudaEventDisableTiming);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&b->ev[k]);
    for (int s = max_jobs - 1; s >= 0; --s) b->free_slots.push_back(s);
    // empty table on the device, step counter zero
    if (e == cudaSuccess) e = b->tab.upload(b->stream);
    if (e == cudaSuccess) e = b->tab.reset_seq(b->stream);
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        (void)cudaGetLastError();
        if (b->h_records) cudaFreeHost(b->h_records);
        if (b->h_live) cudaFreeHost(b->h_live);
        if (b->h_weights) cudaFreeHost(b->h_weights);
        if (b->ev_w) cudaEventDestroy(b->ev_w);
        for (int k = 0; k < 3; ++k)
            if (b->ev[k]) cudaEventDestroy(b->ev[k]);
        delete b;
        return PL_ERR_CUDA;
    }
    b->table_dirty = 0;
    *out = b;
    return PL_OK;
}

PL_API int pl_batch_set_mlp_weights(pl_batch* b, const float* blob, size_t n) {
    if (!b || !blob) return PL_ERR_INVALID_ARG;
    // the blob's length gives the network's input count, which all jobs of a batch share
    const int n_in = n == (size_t)mlp_blob(2) ? 2 : (n == (size_t)mlp_blob(11) ? 11 : 0);
    if (n_in == 0 || (b->mlp_in != 0 && b->mlp_in != n_in)) return PL_ERR_INVALID_ARG;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(blob[k])) return PL_ERR_INVALID_ARG;
    // the pinned staging buffer may still feed the previous upload: wait for that one
    PL_CUDA(cudaEventSynchronize(b->ev_w));
    std::memcpy(b->h_weights, blob, n * sizeof(float));
    float* w32 = reinterpret_cast<float*>(b->base + b->H.w32);
    PL_CUDA(cudaMemcpyAsync(w32, b->h_weights, n * sizeof(float), cudaMemcpyHostToDevice, b->stream));
    PL_CUDA(cudaEventRecord(b->ev_w, b->stream));
    PL_CUDA(launch_convert_weights_bf16(w32, reinterpret_cast<uint16_t*>(b->base + b->H.wbf16), n_in, b->stream));
    b->mlp_in = n_in;
    b->weights_set = 1;
    return PL_OK;
}

PL_API int pl_batch_init_mlp_weights(pl_batch* b, int32_t mlp_in, uint64_t seed) {
    if (!b || (mlp_in != 2 && mlp_in != 11) || (b->mlp_in != 0 && b->mlp_in != mlp_in)) return PL_ERR_INVALID_ARG;
    float* w32 = reinterpret_cast<float*>(b->base + b->H.w32);
    PL_CUDA(launch_init_weights(w32, mlp_in, seed, b->stream));
    PL_CUDA(launch_convert_weights_bf16(w32, reinterpret_cast<uint16_t*>(b->base + b->H.wbf16), mlp_in, b->stream));
    b->mlp_in = mlp_in;
    b->weights_set = 1;
    return PL_OK;
}

PL_API int pl_batch_submit(pl_batch* b, const pl_params* p, const pl_droplet* d, int n, double rho_in, double rho_out,
                           double width, double noise_amp, uint64_t seed, int64_t steps, int64_t* job_id) {
    if (!b || !job_id || steps < 1) return PL_ERR_INVALID_ARG;
    int st = check_params(p);
    if (st) return st;
    if (p->storage != b->storage) return PL_ERR_INVALID_ARG;
    if (b->mlp_in != 0 && p->mlp_in != b->mlp_in) return PL_ERR_INVALID_ARG;  // one network per batch
    if (n < 0 || n > PL_MAX_DROPLETS || (n > 0 && !d) || !(width > 0.0) || !std::isfinite(rho_in) ||
        !std::isfinite(rho_out) || !std::isfinite(noise_amp))
        return PL_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(d[k].cx) || !std::isfinite(d[k].cy) || !(d[k].r >= 0.0)) return PL_ERR_INVALID_ARG;
    // a job occupies a table slot while active and a result slot until polled
    if ((int)(b->jobs.size() + b->pending.size()) >= b->max_jobs) return PL_ERR_BUDGET;
    Job j;
    j.p = *p;
    j.p.mlp = b->mlp;
    j.L = lattice_layout(&j.p);
    j.off = b->arena.alloc(j.L.total);
    if (j.off == SIZE_MAX) return PL_ERR_BUDGET;
    j.id = b->next_id++;
    j.target = (steps + b->K - 1) / b->K * b->K;  // jobs end at an interval boundary
    j.done = 0;
    char* base = b->arena_base + j.off;
    fill_desc(j.desc, &j.p, j.L, base);
    j.desc.phase = b->parity;  // the initial state goes to buffer 0 = phase ^ parity
    j.desc.seq0 = b->steps_total;
    j.desc.has_centre = n == 1;
    j.desc.cx = n == 1 ? d[0].cx : 0.0;
    j.desc.cy = n == 1 ? d[0].cy : 0.0;
    j.desc.width = width;
    // initial state into buffer 0
    LatticeView v{};
    v.nx = p->nx;
    v.ny = p->ny;
    v.storage = p->storage;
    v.pitch = j.L.pitch;
    v.plane = j.L.plane;
    v.pops[0] = j.desc.pops[0];
    v.pops[1] = j.desc.pops[1];
    v.rho = j.desc.rho;
    v.rec = j.desc.rec;
    v.droplets = reinterpret_cast<const pl_droplet*>(b->base + b->H.drops);
    const PhysParams ph{p->G, p->tau, p->rho0, p->mask_eps, p->beta_rho, p->beta_u, p->threshold};
    b->h_drops.assign(d, d + n);
    auto fail = [&](cudaError_t e) {
        g_last_cuda_error = (int)e;
        (void)cudaGetLastError();
        b->arena.release(j.off, j.L.total);
        return PL_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    // the droplet staging is shared: wait for earlier work that reads it, then fill it
    if (n > 0) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(b->base + b->H.drops, b->h_drops.data(), n * sizeof(pl_droplet), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.rec, 0, sizeof(DevRecord), b->stream);
    if (e == cudaSuccess) e = launch_init_droplets(v, ph, 0, n, rho_in, rho_out, width, noise_amp, seed, b->stream);
    if (e != cudaSuccess) return fail(e);
    b->jobs.push_back(j);
    b->mass0_pending = 1;
    if (b->mlp_in == 0) b->mlp_in = p->mlp_in;
    rebuild_table(b);
    *job_id = j.id;
    return PL_OK;
}

PL_API int pl_batch_advance(pl_batch* b, int32_t intervals) {
    if (!b || intervals < 0) return PL_ERR_INVALID_ARG;
    if (!b->weights_set) return PL_ERR_STATE;
    for (int it = 0; it < intervals; ++it) {
        if (b->jobs.empty()) return PL_OK;
        int st = autotune(b, 0);
        if (st) return st;
        st = upload_table(b);
        if (st) return st;
        if (b->mass0_pending) {
            // M0 of newly admitted jobs: metrics of the whole table, keeping the others' M0
            PL_CUDA(launch_metrics_tab(b->tab.view, b->storage, b->parity, 2, 0, b->stream));
            b->mass0_pending = 0;
        }
        const bool capturable =
            b->stream != nullptr && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
        if (!capturable) {
            st = enqueue_interval(b, b->parity, false);
            if (st) return st;
        } else {
            const int gkey = b->parity | (b->tab.edge_lattices > 0 ? 2 : 0);
            auto g = b->graphs.find(gkey);
            if (g == b->graphs.end()) {
                cudaGraph_t graph;
                PL_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const long long before = launches_total();
                st = enqueue_interval(b, b->parity, true);
                const long long captured = launches_total() - before;
                note_launches(-captured);
                cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
                if (st) return st;
                PL_CUDA(ce);
                cudaGraphExec_t ge;
                cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
                cudaGraphDestroy(graph);
                PL_CUDA(ie);
                g = b->graphs.emplace(gkey, GraphEntry{ge, captured}).first;
            }
            PL_CUDA(cudaGraphLaunch(g->second.exec, b->stream));
            note_launches(g->second.kernels);
        }
        b->parity ^= (b->K & 1);
        b->steps_total += (unsigned)b->K;
        // retire finished jobs: copy their records out, free their memory and slots
        std::vector<Job> keep;
        for (auto& j : b->jobs) {
            j.done += b->K;
            if (j.done >= j.target) {
                const int slot = b->free_slots.back();
                b->free_slots.pop_back();
                PL_CUDA(cudaMemcpyAsync(&b->h_records[slot], j.desc.rec, sizeof(DevRecord), cudaMemcpyDeviceToHost,
                                        b->stream));
                pl_batch::Pending pd;
                std::memset(&pd.r, 0, sizeof(pd.r));
                pd.r.id = j.id;
                pd.r.steps = j.done;
                pd.r.nx = j.p.nx;
                pd.r.ny = j.p.ny;
                pd.slot = slot;
                pd.laplace = j.desc.has_centre;
                b->pending.push_back(pd);
                b->arena.release(j.off, j.L.total);  // stream order protects the copy above
            } else {
                keep.push_back(j);
            }
        }
        if (keep.size() != b->jobs.size()) {
            b->jobs.swap(keep);
            rebuild_table(b);
        }
    }
    return PL_OK;
}

PL_API int pl_batch_poll(pl_batch* b, pl_job_result* out, int32_t max, int32_t* n_out) {
    if (!b || !n_out || max < 0 || (max > 0 && !out)) return PL_ERR_INVALID_ARG;
    PL_CUDA(cudaStreamSynchronize(b->stream));
    int n = 0;
    while (n < max && !b->pending.empty()) {
        pl_batch::Pending pd = b->pending.front();
        b->pending.erase(b->pending.begin());
        pl_job_result r = pd.r;
        record_to_metrics(b->h_records[pd.slot], r.nx, r.ny, pd.laplace, &r.metrics);
        r.metrics.step = r.steps;
        r.status = r.metrics.status;
        out[n++] = r;
        b->free_slots.push_back(pd.slot);
    }
    *n_out = n;
    return PL_OK;
}

PL_API int pl_batch_info(pl_batch* b, int32_t* active, int64_t* cells, size_t* arena_used, size_t* arena_total) {
    if (!b) return PL_ERR_INVALID_ARG;
    if (active) *active = (int32_t)b->jobs.size();
    if (cells) *cells = total_cells(b);
    if (arena_used) *arena_used = b->arena.used();
    if (arena_total) *arena_total = b->arena.size();
    return PL_OK;
}

PL_API int pl_batch_get_state(pl_batch* b, int64_t job_id, double* host_f, int64_t* steps) {
    if (!b || !host_f) return PL_ERR_INVALID_ARG;
    for (auto& j : b->jobs) {
        if (j.id != job_id) continue;
        int st = upload_table(b);
        if (st) return st;
        LatticeView v{};
        v.nx = j.p.nx;
        v.ny = j.p.ny;
        v.storage = j.p.storage;
        v.pitch = j.L.pitch;
        v.plane = j.L.plane;
        v.pops[0] = j.desc.pops[0];
        v.pops[1] = j.desc.pops[1];
        v.rho = j.desc.rho;
        v.rec = j.desc.rec;
        const PhysParams ph{j.p.G, j.p.tau, j.p.rho0, j.p.mask_eps, j.p.beta_rho, j.p.beta_u, j.p.threshold};
        const int cur = j.desc.phase ^ b->parity;
        const size_t N = (size_t)j.p.nx * j.p.ny;
        double* staging = static_cast<double*>(j.desc.rho);
        for (int i = 0; i < 9; ++i) {
            PL_CUDA(launch_state_convert(v, ph, cur, staging, i, 1, b->stream));
            PL_CUDA(cudaMemcpyAsync(host_f + (size_t)i * N, staging, N * sizeof(double), cudaMemcpyDeviceToHost,
                                    b->stream));
        }
        PL_CUDA(cudaStreamSynchronize(b->stream));
        if (steps) *steps = j.done;
        return PL_OK;
    }
    return PL_ERR_INVALID_ARG;
}

PL_API int pl_batch_autotune(pl_batch* b, int32_t force, int32_t* rows_per_chunk) {
    if (!b) return PL_ERR_INVALID_ARG;
    int st = autotune(b, force);
    if (st) return st;
    if (rows_per_chunk) *rows_per_chunk = b->rows_per_chunk;
    return PL_OK;
}

PL_API int pl_batch_destroy(pl_batch* b) {
    if (!b) return PL_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->h_records) cudaFreeHost(b->h_records);
    if (b->h_live) cudaFreeHost(b->h_live);
    if (b->h_weights) cudaFreeHost(b->h_weights);
    if (b->ev_w) cudaEventDestroy(b->ev_w);
    for (int k = 0; k < 3; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    delete b;
    return PL_OK;
}

PL_API int pl_batch_interval_times(pl_batch* b, float* steps_ms, float* interval_ms) {
    if (!b) return PL_ERR_INVALID_ARG;
    PL_CUDA(cudaEventSynchronize(b->ev[2]));
    float s = 0.0f, t = 0.0f;
    PL_CUDA(cudaEventElapsedTime(&s, b->ev[0], b->ev[1]));
    PL_CUDA(cudaEventElapsedTime(&t, b->ev[0], b->ev[2]));
    if (steps_ms) *steps_ms = s;
    if (interval_ms) *interval_ms = t;
    return PL_OK;
}

PL_API int pl_batch_metrics(pl_batch* b, pl_job_result* out, int32_t max, int32_t* n_out) {
    if (!b || !n_out || max < 0 || (max > 0 && !out)) return PL_ERR_INVALID_ARG;
    const int n = (int)std::min<size_t>((size_t)max, b->jobs.size());
    for (int k = 0; k < n; ++k)
        PL_CUDA(cudaMemcpyAsync(&b->h_live[k], b->jobs[k].desc.rec, sizeof(DevRecord), cudaMemcpyDeviceToHost,
                                b->stream));
    PL_CUDA(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < n; ++k) {
        const Job& j = b->jobs[k];
        pl_job_result& r = out[k];
        std::memset(&r, 0, sizeof(r));
        r.id = j.id;
        r.steps = j.done;
        r.nx = j.p.nx;
        r.ny = j.p.ny;
        record_to_metrics(b->h_live[k], j.p.nx, j.p.ny, j.desc.has_centre, &r.metrics);
        r.metrics.step = j.done;
        r.status = r.metrics.status;
    }
    *n_out = n;
    return PL_OK;
}

}  // extern "C"
