// common.cuh -- shared helpers of the GB300 FMM library (CUDA path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/fmm.h"

namespace fmm {

// Tree keys: 21 bits per axis, interleaved x,y,z -> 63-bit Morton key.
constexpr int kKeyBits = 21;
constexpr int kMaxLevel = 21;
// Targets per M2L GEMM tile (one tile = the children with a common octant of
// up to kTile consecutive split parents).
constexpr int kTile = 128;

// Status carried through the host orchestration.
struct Error {
    fmm_status code;
    std::string msg;
};

void set_last_error(const std::string &msg);

#define FMM_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess) {                                                             \
            throw ::fmm::Error{FMM_ERR_CUDA, std::string(#expr) + ": " +                     \
                                                 cudaGetErrorString(_e) + " at " + __FILE__ + \
                                                 ":" + std::to_string(__LINE__)};            \
        }                                                                                    \
    } while (0)

// Every kernel launch is followed by this check, which also counts it.
extern thread_local int64_t g_launch_count;
#define FMM_LAUNCH_CHECK()                   \
    do {                                     \
        ++::fmm::g_launch_count;             \
        FMM_CUDA_TRY(cudaGetLastError());    \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Raises a kernel's dynamic shared memory limit once per device and value
// (cudaFuncSetAttribute may synchronise, so it stays out of the per-solve path).
void set_smem_limit_once(const void *func, int bytes);
// Sets a kernel's preferred L1/shared carveout once per device.
void set_carveout_once(const void *func, int carveout);
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// (p+1)^2 real coefficients, padded to a multiple of 32.
__host__ __device__ inline int nterms(int p) { return (p + 1) * (p + 1); }
inline int nterms_pad(int p) { return (int)round_up(nterms(p), 32); }

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ uint64_t spread3_dev(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3_dev(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// Integer geometry of a cell: centre in units of side/2^22 (always an odd
// multiple of the half side) and half side.
__device__ __forceinline__ void cell_int_geom(int level, uint64_t prefix, int64_t C[3], int64_t &h)
{
    h = (int64_t)1 << (kKeyBits - level);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int64_t k = compact3_dev(prefix >> a);
        C[a] = (2 * k + 1) * h;
    }
}

// ---------------------------------------------------------------- scan

// Exclusive prefix sum of n values; *total_dev (if non-null) receives the sum.
// temp must hold scan_temp_elems(n) values.
template <typename T>
void scan_exclusive(const T *in, T *out, int64_t n, T *total_dev, T *temp, cudaStream_t st);
int64_t scan_temp_elems(int64_t n);

// ---------------------------------------------------------------- radix sort

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the key
// (8-bit digits).  keys/vals are sorted in place (alt buffers are scratch of the
// same size).  scratch must hold radix_scratch_elems(n) uint32 values.  flags
// (nullable) receives kFlagTimeout if a bounded wait of the look-back expires.
constexpr int kRadixTile = 4096;     // keys per block
constexpr int kRadixMaxPasses = 8;   // 64-bit keys
constexpr int64_t radix_scratch_elems(int64_t n)
{
    // digit counts of every pass, tile counters, then per pass and tile 256
    // 64-bit look-back words
    return (int64_t)kRadixMaxPasses * 256 + 64 +
           (int64_t)kRadixMaxPasses * 256 * 2 * ((n + kRadixTile - 1) / kRadixTile);
}
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, uint32_t *scratch, int *flags, cudaStream_t st);

}  // namespace fmm
