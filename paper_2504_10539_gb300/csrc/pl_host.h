// Host-side runtime pieces shared by the single-lattice and the batch ABI:
// argument checks, the per-lattice memory layout, and the job table (host mirror
// of the device-resident table the kernels read).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pinnlbm.h"
#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

extern thread_local int g_last_cuda_error;

// On failure: remember the error for pl_last_cuda_error() and clear the runtime's
// last-error slot so that it does not surface in a later call.
#define PL_CUDA(call)                        \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) {             \
            ::pl::g_last_cuda_error = (int)e_; \
            (void)cudaGetLastError();        \
            return PL_ERR_CUDA;              \
        }                                    \
    } while (0)

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }
inline size_t storage_bytes(int storage) { return storage == PL_F64 ? 8 : (storage == PL_F32 ? 4 : 2); }
inline size_t scratch_elem_bytes(int storage) { return storage == PL_F64 ? 8 : 4; }
// Stored rows are padded to a multiple of 8 populations so that every row, and every
// even column pair, is aligned for vector access.
inline int row_pitch(int nx) { return (nx + 7) / 8 * 8; }

// FP32 weight blob: W1[64 x n_in] b1 W2 b2 W3 b3 W4 b4 W5 b5 (n_in = 2 or 11)
constexpr int mlp_blob(int n_in) {
    return 64 * n_in + 64 + 128 * 64 + 128 + 128 * 128 + 128 + 64 * 128 + 64 + 3 * 64 + 3;
}
constexpr int MLP_BLOB = mlp_blob(2);
constexpr int MLP_BLOB_MAX = mlp_blob(11);  // the size every weight buffer is laid out for

int check_params(const pl_params* p);

// Device memory of one lattice (populations, scratch, partials, record).
struct LatLayout {
    size_t pops[2], scratch, partials, rec, total;
    int pitch;
    long long plane;
    int red_blocks;
};
LatLayout lattice_layout(const pl_params* p);

// Fill a descriptor for a lattice placed at `base` (layout L).
void fill_desc(LatDesc& d, const pl_params* p, const LatLayout& L, char* base);

// Job table: host mirror + device region (header, descriptors, prefix sums, step counter).
struct Table {
    int cap = 0;
    char* dev = nullptr;
    TableView view{};
    std::vector<LatDesc> d;
    std::vector<char> staging;  // host image of the device region
    long long total_warps = 0, total_tiles = 0;
    int total_blocks = 0;
    int edge_lattices = 0;      // FP16 lattices off the step's vector path (k_step_edge's work)

    static size_t bytes(int cap);
    void carve(char* base, int capacity);
    // Recompute prefix sums for the first n descriptors and copy everything but the step
    // counter to the device on stream s.
    cudaError_t upload(cudaStream_t s);
    cudaError_t reset_seq(cudaStream_t s);
};

// Device record -> public metric record (Eqs. 9-15, Laplace fields if `laplace`).
void record_to_metrics(const DevRecord& r, int nx, int ny, int laplace, pl_metric_record* out);

// Step decomposition of a lattice given a target number of rows per chunk.
void set_chunks(LatDesc& d, int rows_per_chunk);
// Single-lattice decomposition: as many row chunks as keep every warp resident.
void set_chunks_single(LatDesc& d, int storage);

}  // namespace pl
