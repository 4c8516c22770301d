// noalloc.cu -- the by-cell counting sort of pic_compact as a standalone
// operation on caller buffers that allocates no device memory.
//
// Why it exists: pic_compact keeps its per-cell counts and offsets in memory
// that pic_create allocates.  Code that must not call cudaMalloc (a host
// framework that owns every allocation, a memory pool that must not grow, a
// process that has reserved all device memory) can still sort a particle set
// by cell with pic_op_sort_noalloc: its only scratch is the file-scope
// __device__ array below, part of the library image, so it costs 32 KiB per
// GPU on which the library is loaded and is never freed.
//
// Because every call shares that one array:
//   - each call clears the per-cell counts first (the array keeps the last
//     call's contents; the running offsets are rewritten by the scan);
//   - calls whose work overlaps on the GPU -- on different streams, or from
//     different host threads on one device -- race on the array and give
//     wrong results; the caller must order them (one stream, or events).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/pic_gb300.h"
#include "launch.h"

using namespace pg;

namespace {

constexpr int kNoAllocMaxCells = 4096;   // largest n_cells the static scratch holds
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxCells): per-cell counts; [kNoAllocMaxCells, 2 kNoAllocMaxCells): running offsets
static __device__ __align__(256) unsigned int g_sort_scratch[2 * kNoAllocMaxCells];

struct DevEntry {
    unsigned int* scratch;
    int sms;
};
std::mutex g_mu;
DevEntry g_dev[kMaxDevices] = {};

template <typename PosT>
__global__ void k_na_count(const PosT* __restrict__ pos, long long n, int ncell, int kshift, unsigned int* cnt)
{
    extern __shared__ unsigned int hist[];
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const PosT x = pos[i];
        if (!is_alive(x)) continue;
        uint32_t j, wr;
        cell_of(x, kshift, j, wr);
        if (j < (uint32_t)ncell) atomicAdd(&hist[j], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncell; i += blockDim.x)
        if (hist[i]) atomicAdd(&cnt[i], hist[i]);
}

// Exclusive scan of the counts into the running offsets; one CTA of 1024
// threads, each owning a contiguous run of ceil(ncell / 1024) cells.
__global__ void k_na_scan(int ncell, const unsigned int* cnt, unsigned int* off, int64_t* n_out)
{
    __shared__ unsigned int part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int seg = (ncell + T - 1) / T;
    const int m0 = min(t * seg, ncell), m1 = min(m0 + seg, ncell);
    unsigned int a = 0;
    for (int m = m0; m < m1; ++m) a += cnt[m];
    part[t] = a;
    __syncthreads();
    for (int k = 1; k < T; k <<= 1) {   // inclusive scan of the per-thread totals
        const unsigned int y = t >= k ? part[t - k] : 0u;
        __syncthreads();
        part[t] += y;
        __syncthreads();
    }
    unsigned int o = part[t] - a;
    for (int m = m0; m < m1; ++m) {
        off[m] = o;
        o += cnt[m];
    }
    if (t == T - 1 && n_out) *n_out = (int64_t)part[T - 1];
}

// Scatter: lanes of a warp that share a cell take consecutive slots with one
// atomic on that cell's running offset.
template <typename PosT>
__global__ void k_na_scatter(const PosT* __restrict__ pos, const float* __restrict__ vx,
                             const float* __restrict__ vy, const float* __restrict__ vz,
                             const uint64_t* __restrict__ id, long long n, int ncell, int kshift,
                             unsigned int* off, PosT* pos_o, float* vx_o, float* vy_o, float* vz_o,
                             uint64_t* id_o)
{
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nround = (n + stride - 1) / stride * stride;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nround; i += stride) {
        bool act = i < n;
        PosT x = 0;
        if (act) {
            x = pos[i];
            act = is_alive(x);
        }
        uint32_t j = 0xffffffffu, wr;
        if (act) {
            cell_of(x, kshift, j, wr);
            if (j >= (uint32_t)ncell) {
                act = false;
                j = 0xffffffffu;
            }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1u));
        unsigned int base = 0;
        if (act && lane == leader) base = atomicAdd(&off[j], (unsigned)__popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (act) {
            const unsigned int o = base + rank;
            pos_o[o] = x;
            vx_o[o] = vx[i];
            vy_o[o] = vy[i];
            vz_o[o] = vz[i];
            id_o[o] = id[i];
        }
    }
}

// The scratch array's device address and the SM count of the current device.
// The address is looked up on every call (a host-side query once the
// library's module is loaded on the device): a device reset or a new primary
// context reloads the module, and an address kept from before would then
// point at freed memory.  The first call on a device loads the module, so it
// should come before any stream capture.  The SM count is kept per ordinal.
int device_entry(DevEntry* out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return PIC_ERR_NO_DEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("device ordinal above the no-alloc sort's device table");
        return PIC_ERR_INVALID_ARG;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p) {
        set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress gave NULL");
        return PIC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    DevEntry& d = g_dev[dev];
    if (d.sms < 1) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms < 1) {
            set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "no multiprocessors");
            return PIC_ERR_CUDA;
        }
        d.sms = sms;
    }
    d.scratch = (unsigned int*)p;
    *out = d;
    return PIC_OK;
}

}  // namespace

extern "C" int pic_op_sort_noalloc(int pos_precision, int64_t n, int32_t n_cells, const void* pos,
                                   const float* vx, const float* vy, const float* vz, const uint64_t* id,
                                   void* pos_out, float* vx_out, float* vy_out, float* vz_out,
                                   uint64_t* id_out, int64_t* n_out, void* stream)
{
    if (n_cells < 4 || n_cells > kNoAllocMaxCells || (n_cells & (n_cells - 1))) {
        set_last_error("n_cells must be a power of two in [4, 4096], the size of the static scratch");
        return PIC_ERR_INVALID_ARG;
    }
    if (pos_precision != 32 && pos_precision != 64) {
        set_last_error("pos_precision must be 32 or 64");
        return PIC_ERR_INVALID_ARG;
    }
    if (n < 0 || n > 0xffffffffll) {
        set_last_error("n must be in [0, 2^32 - 1]");
        return PIC_ERR_INVALID_ARG;
    }
    if (n > 0 && (!pos || !vx || !vy || !vz || !id || !pos_out || !vx_out || !vy_out || !vz_out || !id_out)) {
        set_last_error("NULL particle buffer");
        return PIC_ERR_INVALID_ARG;
    }
    DevEntry d;
    int rc = device_entry(&d);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int kshift = 0;
    while ((1 << kshift) < n_cells) ++kshift;
    unsigned int* cnt = d.scratch;
    unsigned int* off = d.scratch + kNoAllocMaxCells;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * n_cells, st);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    const long long want = (n + 2047) / 2048;
    const int grid = (int)(want < 1 ? 1 : (want > 4ll * d.sms ? 4ll * d.sms : want));
    const size_t hs = sizeof(unsigned int) * n_cells;
    if (pos_precision == 32) {
        k_na_count<uint32_t><<<grid, 256, hs, st>>>((const uint32_t*)pos, n, n_cells, kshift, cnt);
        k_na_scan<<<1, 1024, 0, st>>>(n_cells, cnt, off, n_out);
        k_na_scatter<uint32_t><<<grid, 256, 0, st>>>((const uint32_t*)pos, vx, vy, vz, id, n, n_cells, kshift,
                                                     off, (uint32_t*)pos_out, vx_out, vy_out, vz_out, id_out);
    } else {
        k_na_count<double><<<grid, 256, hs, st>>>((const double*)pos, n, n_cells, kshift, cnt);
        k_na_scan<<<1, 1024, 0, st>>>(n_cells, cnt, off, n_out);
        k_na_scatter<double><<<grid, 256, 0, st>>>((const double*)pos, vx, vy, vz, id, n, n_cells, kshift, off,
                                                   (double*)pos_out, vx_out, vy_out, vz_out, id_out);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}
