// Morton sort of a body set without any device allocation.
//
// fmm_morton_sort_noalloc computes the bounding cube and the 63-bit Morton
// keys of up to kNoAllocMaxN bodies and sorts them with their indices: the
// same keys and permutation that fmm_solve builds its octree from. Its
// scratch (block partials of the bounding box, the second key buffer of the
// radix sort, the index buffers and the digit histograms) lives in one
// file-scope device array, so the call allocates nothing.
//
// It exists for callers that cannot call cudaMalloc while they work: code
// that runs under a device-memory budget owned by another allocator (a
// framework's caching allocator, a real-time loop that forbids allocation
// after start-up), or that cannot afford an allocation's latency or failure
// inside its loop. The price is that every GPU that loads this library holds
// the array (kNoAllocScratchBytes, about 4.3 MB) until the process exits.
//
// Compiled with -fmad=false, like the tree build, so the keys are bit for bit
// those of fmm_solve.
#include <mutex>

#include "gbfmm_internal.cuh"

namespace gbfmm {
void set_global_error(const char* msg);

namespace {

constexpr int64_t kNoAllocMaxN = 262144;  // bodies per call at most
constexpr int kBboxBlocks = 304;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int64_t kMaxSortBlocks = (kNoAllocMaxN + 4095) / 4096;  // radix-sort tiles of 4096 keys
constexpr size_t kHistWords = 256 * kMaxSortBlocks + 1 + (256 * kMaxSortBlocks + 4095) / 4096 + 2;
constexpr size_t kOffScalars = 0;
constexpr size_t kOffBbox = align256(kOffScalars + sizeof(DevScalars));
constexpr size_t kOffAltKeys = align256(kOffBbox + 6 * kBboxBlocks * sizeof(double));
constexpr size_t kOffIdx0 = align256(kOffAltKeys + kNoAllocMaxN * sizeof(uint64_t));
constexpr size_t kOffIdx1 = align256(kOffIdx0 + kNoAllocMaxN * sizeof(uint32_t));
constexpr size_t kOffHist = align256(kOffIdx1 + kNoAllocMaxN * sizeof(uint32_t));
constexpr size_t kNoAllocScratchBytes = align256(kOffHist + kHistWords * sizeof(uint32_t));

// The scratch of every call: one array per device, shared by all calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Its device address, looked up once per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
std::mutex g_mu;
void* g_scratch_addr[64] = {};

__global__ void k_na_bbox_partial(const double* __restrict__ x, const double* __restrict__ y,
                                  const double* __restrict__ z, int64_t n, double* __restrict__ part,
                                  unsigned* err) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!isfinite(v[d])) bad = true;
            mn[d] = fmin(mn[d], v[d]);
            mx[d] = fmax(mx[d], v[d]);
        }
    }
    __shared__ double s[6][256];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
    if (bad) atomicOr(err, kErrNonfinite);
}

// cube centre (min+max)/2, half-size the largest (max-min)/2 (1 if zero)
__global__ void k_na_bbox_final(const double* __restrict__ part, int nparts, DevScalars* ds) {
    if (threadIdx.x != 0) return;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nparts; ++b)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], part[6 * b + d]);
            mx[d] = fmax(mx[d], part[6 * b + 3 + d]);
        }
    double h = 0.0;
    for (int d = 0; d < 3; ++d) {
        ds->box[d] = 0.5 * (mn[d] + mx[d]);
        const double hd = 0.5 * (mx[d] - mn[d]);
        if (hd > h) h = hd;
    }
    if (h == 0.0) h = 1.0;
    ds->box[3] = h;
    for (int d = 0; d < 3; ++d) ds->box[4 + d] = ds->box[d] - h;
    ds->box[7] = 2.0 * h;
}

__device__ __forceinline__ uint64_t na_spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t na_quantise(double v, double lo, double size) {
    const double t = (v - lo) / size;
    double f = floor(t * 2097152.0);
    f = f < 0.0 ? 0.0 : (f > 2097151.0 ? 2097151.0 : f);
    return (uint64_t)f;
}

__global__ void k_na_keys(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                          int64_t n, const DevScalars* __restrict__ ds, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double size = ds->box[7];
    keys[i] = (na_spread3(na_quantise(x[i], ds->box[4], size)) << 2) |
              (na_spread3(na_quantise(y[i], ds->box[5], size)) << 1) | na_spread3(na_quantise(z[i], ds->box[6], size));
    idx[i] = (uint32_t)i;
}

__global__ void k_na_perm64(const uint32_t* __restrict__ idx, int64_t n, int64_t* __restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int64_t)idx[i];
}

}  // namespace
}  // namespace gbfmm

using namespace gbfmm;

extern "C" int fmm_morton_sort_noalloc(int64_t n, const double* x, const double* y, const double* z,
                                       uint64_t* keys, int64_t* perm, double* box, void* cuda_stream) {
    if (n < 0 || n > kNoAllocMaxN) {
        set_global_error("fmm_morton_sort_noalloc: n must be in [0, 262144] (its static scratch holds that many bodies)");
        return FMM_ERR_ARG;
    }
    if (n == 0) return FMM_OK;
    if (!x || !y || !z || !keys || !perm) {
        set_global_error("fmm_morton_sort_noalloc: NULL input or output pointer");
        return FMM_ERR_ARG;
    }
    if (radix_hist_words(n) > kHistWords) {
        set_global_error("fmm_morton_sort_noalloc: histogram scratch too small");
        return FMM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        set_global_error("fmm_morton_sort_noalloc: no usable CUDA device");
        return FMM_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* addr = nullptr;
            const cudaError_t rc = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (rc != cudaSuccess || !addr) {
                cudaGetLastError();
                set_global_error("fmm_morton_sort_noalloc: cudaGetSymbolAddress of the static scratch failed");
                return FMM_ERR_CUDA;
            }
            g_scratch_addr[dev] = addr;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevScalars* ds = reinterpret_cast<DevScalars*>(base + kOffScalars);
    double* part = reinterpret_cast<double*>(base + kOffBbox);
    uint64_t* alt = reinterpret_cast<uint64_t*>(base + kOffAltKeys);
    uint32_t* idx0 = reinterpret_cast<uint32_t*>(base + kOffIdx0);
    uint32_t* idx1 = reinterpret_cast<uint32_t*>(base + kOffIdx1);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    // the array keeps the previous call's contents: clear the error word
    if (cudaMemsetAsync(&ds->err, 0, sizeof(unsigned), st) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("fmm_morton_sort_noalloc: cudaMemsetAsync failed");
        return FMM_ERR_CUDA;
    }
    k_na_bbox_partial<<<kBboxBlocks, 256, 0, st>>>(x, y, z, n, part, &ds->err);
    k_na_bbox_final<<<1, 32, 0, st>>>(part, kBboxBlocks, ds);
    const int nb = (int)((n + 255) / 256);
    k_na_keys<<<nb, 256, 0, st>>>(x, y, z, n, ds, keys, idx0);
    const int in1 = radix_sort(keys, idx0, alt, idx1, n, 63, hist, st);
    if (in1 && cudaMemcpyAsync(keys, alt, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("fmm_morton_sort_noalloc: key copy failed");
        return FMM_ERR_CUDA;
    }
    k_na_perm64<<<nb, 256, 0, st>>>(in1 ? idx1 : idx0, n, perm);
    if (box && cudaMemcpyAsync(box, ds->box, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("fmm_morton_sort_noalloc: box copy failed");
        return FMM_ERR_CUDA;
    }
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, &ds->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaGetLastError();
        set_global_error("fmm_morton_sort_noalloc: a CUDA call failed");
        return FMM_ERR_CUDA;
    }
    if (err & kErrNonfinite) {
        set_global_error("fmm_morton_sort_noalloc: non-finite position");
        return FMM_ERR_NONFINITE;
    }
    return FMM_OK;
}
