// noalloc.cu -- Morton keys and sorted order without any device allocation.
//
// fmm_laplace3d grows a device workspace with cudaMalloc on first use and
// whenever a problem is larger than any before.  Some callers cannot allow
// that: code that runs while another framework owns device memory through its
// own pool (a cudaMalloc there can fail, or synchronise the whole device and
// stall everyone else's streams), or a host that only lets plugins allocate
// during initialisation.  For them this file offers the first stage of the
// solve -- bounding box, FP64 quantisation, 63-bit Morton keys and the stable
// radix sort -- with every scratch array inside one fixed, file-scope device
// array.  The caller passes the inputs and the output buffers.
//
// The scratch holds the sort's second key/index buffers, digit counts and
// look-back words, the box and the flags for up to kNoAllocMaxN points.  It is
// resolved to a device address with cudaGetSymbolAddress once per device, on
// that device's first call.  Under lazy module loading (CUDA's default) the
// array itself is placed in device memory at that first use of the module on
// the device, so the first call per device belongs in the caller's
// initialisation.  All calls share it and it keeps the previous call's
// contents; everything that must start at zero is cleared on every call.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr int64_t kHistElems = radix_scratch_elems(kNoAllocMaxN);
constexpr size_t kOffKeysAlt = 0;
constexpr size_t kOffIdxAlt = align256(kOffKeysAlt + sizeof(uint64_t) * kNoAllocMaxN);
constexpr size_t kOffHist = align256(kOffIdxAlt + sizeof(uint32_t) * kNoAllocMaxN);
constexpr size_t kOffBbox = align256(kOffHist + sizeof(uint32_t) * kHistElems);
constexpr size_t kOffFlags = align256(kOffBbox + sizeof(uint32_t) * 6);
constexpr size_t kScratchBytes = align256(kOffFlags + sizeof(int) * kNumFlags);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};

// Device address of the scratch array for the current device (set-up on the
// device's first call).
unsigned char *scratch_for_current_device()
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{FMM_ERR_ARG, "device ordinal out of range"};
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        FMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    return static_cast<unsigned char *>(g_noalloc_addr[dev]);
}

}  // namespace

}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_morton_sort_noalloc(const float *xyz, int64_t N, uint64_t *keys,
                                              int32_t *order, double *box, void *stream)
{
    try {
        if (!xyz || !keys || !order || !box) throw Error{FMM_ERR_ARG, "null pointer argument"};
        if (N < 1) throw Error{FMM_ERR_ARG, "N must be >= 1"};
        if (N > kNoAllocMaxN)
            throw Error{FMM_ERR_ARG, "N exceeds the fixed scratch of fmm_morton_sort_noalloc (at most "
                                         "1048576 points)"};
        cudaStream_t st = (cudaStream_t)stream;
        unsigned char *s = scratch_for_current_device();
        uint64_t *keys_alt = reinterpret_cast<uint64_t *>(s + kOffKeysAlt);
        uint32_t *idx_alt = reinterpret_cast<uint32_t *>(s + kOffIdxAlt);
        uint32_t *hist = reinterpret_cast<uint32_t *>(s + kOffHist);
        uint32_t *bbox_u = reinterpret_cast<uint32_t *>(s + kOffBbox);
        int *flags = reinterpret_cast<int *>(s + kOffFlags);
        uint32_t *idx = reinterpret_cast<uint32_t *>(order);
        FMM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * kNumFlags, st));
        FMM_CUDA_TRY(cudaMemsetAsync(bbox_u, 0xff, 3 * sizeof(uint32_t), st));
        FMM_CUDA_TRY(cudaMemsetAsync(bbox_u + 3, 0, 3 * sizeof(uint32_t), st));
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(N, 256), 152 * 16);
        k_bbox<<<grid, 256, 0, st>>>(xyz, N, bbox_u, flags);
        FMM_LAUNCH_CHECK();
        k_morton<<<grid, 256, 0, st>>>(xyz, N, nullptr, 1, bbox_u, box, keys, idx);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(keys, idx, keys_alt, idx_alt, N, 63, hist, flags, st);
        int hflags[kNumFlags];
        FMM_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
        if (hflags[kFlagNonfinite]) throw Error{FMM_ERR_NONFINITE, "a coordinate is NaN or infinite"};
        if (hflags[kFlagTimeout]) throw Error{FMM_ERR_TIMEOUT, "a bounded device-side wait expired (radix sort)"};
        set_last_error("");
        return FMM_OK;
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("unexpected exception");
        return FMM_ERR_CUDA;
    }
}
