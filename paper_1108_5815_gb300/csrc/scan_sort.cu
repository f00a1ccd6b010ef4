// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both are building blocks of the tree construction (sorting Morton keys, the
// paper's tree build which it ran on the host CPU) and of the list compaction
// in the dual tree traversal.  Written for coalesced HBM access: each block
// owns a contiguous tile, and the radix scatter reorders a whole tile in shared
// memory first so that each digit's run is written contiguously.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

template <typename T>
__device__ __forceinline__ T warp_inclusive(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the block total via *total.
template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T *smem_warp, T *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T inc = warp_inclusive(v);
    if (lane == 31) smem_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? smem_warp[lane] : T(0);
        T wi = warp_inclusive(w);
        if (lane < nwarps) smem_warp[lane] = wi - w;
        if (lane == nwarps - 1) smem_warp[32] = wi;
    }
    __syncthreads();
    T res = inc - v + smem_warp[warp];
    *total = smem_warp[32];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ sums)
{
    __shared__ T sw[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    T tot;
    block_exclusive(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Scans `n` values (any n) with a single block, chunk by chunk with a carry.
template <typename T>
__global__ void k_scan_single(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                              T *__restrict__ total)
{
    __shared__ T sw[33];
    T carry = 0;
    for (int64_t base = 0; base < n; base += kScanTile) {
        T v[kScanItems];
        T s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
            v[i] = idx < n ? in[idx] : T(0);
            s += v[i];
        }
        T tot;
        T ex = block_exclusive(s, sw, &tot);
        ex += carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
            if (idx < n) out[idx] = ex;
            ex += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_tile_scan(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            const T *__restrict__ offs)
{
    __shared__ T sw[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = idx < n ? in[idx] : T(0);
        s += v[i];
    }
    T tot;
    T ex = block_exclusive(s, sw, &tot) + offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = ex;
        ex += v[i];
    }
}

}  // namespace

int64_t scan_temp_elems(int64_t n) { return 2 * ceil_div(n, kScanTile) + 2; }

template <typename T>
void scan_exclusive(const T *in, T *out, int64_t n, T *total_dev, T *temp, cudaStream_t st)
{
    if (n <= 0) {
        if (total_dev) FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(T), st));
        return;
    }
    if (n <= 4 * kScanTile) {
        k_scan_single<T><<<1, kScanThreads, 0, st>>>(in, out, n, total_dev);
        FMM_LAUNCH_CHECK();
        return;
    }
    const int64_t tiles = ceil_div(n, kScanTile);
    T *sums = temp, *offs = temp + tiles;
    k_tile_reduce<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums);
    FMM_LAUNCH_CHECK();
    k_scan_single<T><<<1, kScanThreads, 0, st>>>(sums, offs, tiles, total_dev);
    FMM_LAUNCH_CHECK();
    k_tile_scan<T><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, offs);
    FMM_LAUNCH_CHECK();
}

template void scan_exclusive<int32_t>(const int32_t *, int32_t *, int64_t, int32_t *, int32_t *,
                                      cudaStream_t);
template void scan_exclusive<uint32_t>(const uint32_t *, uint32_t *, int64_t, uint32_t *,
                                       uint32_t *, cudaStream_t);
template void scan_exclusive<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, int64_t *,
                                      cudaStream_t);

// ---------------------------------------------------------------- radix sort
//
// One kernel per 8-bit digit (a one-sweep LSD sort, after Adinets & Merrill,
// "Onesweep", 2022): the digit counts of every pass come from one read of the
// keys before the first pass; in a pass each block takes the next tile of 4096
// keys from a counter, ranks them stably in shared memory, publishes its
// per-digit counts, and adds the counts of the tiles before it by looking back
// over their published words (a tile that has finished its own look-back
// publishes its inclusive prefix, which ends the walk).  Blocks take tiles in
// the order they start, so every tile a block waits for belongs to a block
// that has started and never waits for a later tile; each wait is bounded
// anyway and reports kFlagTimeout if it runs out.

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = kRadixTile / kSortThreads;  // 16
constexpr int kSortTile = kRadixTile;
constexpr int kRadix = 256;
constexpr uint64_t kLbAggregate = 1ull << 62;  // look-back word: tile count only
constexpr uint64_t kLbInclusive = 2ull << 62;  // look-back word: prefix through this tile
constexpr uint32_t kLookbackPolls = 1u << 20;
constexpr int kLookbackWindow = 8;  // earlier tiles whose look-back words are read together

// The lanes of the warp whose 8-bit digit equals this lane's: one ballot per
// digit bit, each keeping the lanes that agree on that bit.
__device__ __forceinline__ unsigned digit_peers(uint32_t dig)
{
    unsigned peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (dig >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// Digit counts of passes 0 .. passes-1 over all keys (counts[pass][digit], zeroed).
__global__ void __launch_bounds__(256)
    k_radix_counts(const uint64_t *__restrict__ keys, int64_t n, int passes, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t h[kRadixMaxPasses * kRadix];
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kRadix + ((k >> (8 * p)) & 0xff)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}

// One pass: stable scatter of one tile by the digit at `shift`.  The tile is
// ranked (index order), reordered in shared memory by digit, and each digit's
// run is written contiguously at the digit's global start plus the keys of that
// digit in earlier tiles.
__global__ void __launch_bounds__(kSortThreads, 2)
    k_radix_pass(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                 uint32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ counts,
                 unsigned long long *status, int *tile_counter, int *flags)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);                 // kSortTile keys
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);           // kSortTile vals
    uint32_t *wcnt = sv + kSortTile;                                       // [8 warps][256]
    uint32_t *run = wcnt + 8 * kRadix;                                     // [256] running count
    uint32_t *tile_off = run + kRadix;                                     // [256]
    uint32_t *gbase = tile_off + kRadix;                                   // [256]
    uint32_t *sw = gbase + kRadix;                                         // [33] scan scratch
    __shared__ int s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
    run[tid] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * kSortTile;
    const int tile_n = (int)(n - base < (int64_t)kSortTile ? n - base : (int64_t)kSortTile);
    uint32_t gtot;
    const uint32_t gstart = block_exclusive<uint32_t>(counts[tid], sw, &gtot);  // digit tid's global start
    const unsigned lt_mask = (1u << lane) - 1u;

    // Warp w holds the tile's keys w * 512 .. w * 512 + 511 (item i of lane l at
    // w * 512 + 32 i + l) and ranks them in index order with warp-private digit
    // counters; one prefix over the 8 warps per digit then makes the ranks
    // tile-wide.  Equal digits keep their index order (stable).
    constexpr int kWarpKeys = kSortItems * 32;
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = warp * kWarpKeys + i * 32 + lane;
        const bool valid = li < tile_n;
        key[i] = valid ? kin[base + li] : ~0ull;
        val[i] = valid ? vin[base + li] : 0u;
    }
    for (int d = tid; d < 8 * kRadix; d += kSortThreads) wcnt[d] = 0;
    __syncthreads();
    uint32_t *wc = wcnt + warp * kRadix;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = warp * kWarpKeys + i * 32 + lane;
        const bool valid = li < tile_n;
        const uint32_t dig = (uint32_t)(key[i] >> shift) & 0xffu;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        const unsigned peers = digit_peers(dig) & active;
        const uint32_t lr = __popc(peers & lt_mask);
        rank[i] = valid ? wc[dig] + lr : 0u;
        __syncwarp();
        if (valid && lr == 0) wc[dig] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the 8 warps; run[] = the tile's count
    {
        const int d = tid;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = wcnt[w * kRadix + d];
            wcnt[w * kRadix + d] = acc;
            acc += c;
        }
        run[d] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = warp * kWarpKeys + i * 32 + lane;
        if (li < tile_n) rank[i] += wc[(uint32_t)(key[i] >> shift) & 0xffu];
    }

    // this tile's count of digit tid, published; then the earlier tiles' counts
    {
        const uint32_t cnt = run[tid];
        volatile unsigned long long *mine = status + (int64_t)tile * kRadix + tid;
        uint32_t excl = 0;
        if (tile == 0) {
            *mine = kLbInclusive | cnt;
        } else {
            *mine = kLbAggregate | cnt;
            // The words of the next kLookbackWindow earlier tiles are read together
            // (independent loads), then taken in order: the walk costs one memory
            // latency per window, not per tile.
            bool done = false;
            for (int t0 = tile - 1; t0 >= 0 && !done; t0 -= kLookbackWindow) {
                unsigned long long v[kLookbackWindow];
#pragma unroll
                for (int j = 0; j < kLookbackWindow; ++j)
                    v[j] = t0 - j >= 0 ? *(volatile unsigned long long *)(status + (int64_t)(t0 - j) * kRadix + tid) : 0ull;
#pragma unroll
                for (int j = 0; j < kLookbackWindow; ++j) {
                    if (done || t0 - j < 0) break;
                    volatile unsigned long long *pv = status + (int64_t)(t0 - j) * kRadix + tid;
                    uint32_t polls = 0;
                    while ((v[j] >> 62) == 0 && polls < kLookbackPolls) {
                        __nanosleep(32);
                        v[j] = *pv;
                        ++polls;
                    }
                    if ((v[j] >> 62) == 0) {  // gave up: the result of this sort is invalid
                        if (flags) atomicOr(&flags[kFlagTimeout], 1);
                        done = true;
                        break;
                    }
                    excl += (uint32_t)(v[j] & 0xffffffffull);
                    if ((v[j] >> 62) == 2) done = true;
                }
            }
            *mine = kLbInclusive | (excl + cnt);
        }
        gbase[tid] = gstart + excl;
    }
    // tile-level digit offsets (exclusive scan of run[] over digits)
    {
        uint32_t tot;
        const uint32_t ex = block_exclusive<uint32_t>(run[tid], sw, &tot);
        tile_off[tid] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = warp * kWarpKeys + i * 32 + lane;
        if (li < tile_n) {
            const uint32_t dig = (uint32_t)(key[i] >> shift) & 0xffu;
            const uint32_t pos = tile_off[dig] + rank[i];
            sk[pos] = key[i];
            sv[pos] = val[i];
        }
    }
    __syncthreads();
    for (int li = tid; li < tile_n; li += kSortThreads) {
        const uint64_t k = sk[li];
        const uint32_t dig = (uint32_t)(k >> shift) & 0xffu;
        const int64_t dst = (int64_t)gbase[dig] + (li - (int)tile_off[dig]);
        if (dst < n) {  // always, unless a wait gave up
            kout[dst] = k;
            vout[dst] = sv[li];
        }
    }
}

constexpr size_t kPassSmem = (size_t)kSortTile * 8 + (size_t)kSortTile * 4 + (8 * kRadix + 3 * kRadix + 33) * 4;

}  // namespace

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, uint32_t *scratch, int *flags, cudaStream_t st)
{
    if (n <= 1) return;
    set_smem_limit_once((const void *)k_radix_pass, (int)kPassSmem);
    const int64_t ntiles = ceil_div(n, kSortTile);
    const int passes = (int)std::min<int64_t>(kRadixMaxPasses, ceil_div(bits, 8));
    uint32_t *counts = scratch;                                        // [passes][256]
    int *tile_counter = reinterpret_cast<int *>(scratch + kRadixMaxPasses * kRadix);  // [passes]
    unsigned long long *status =
        reinterpret_cast<unsigned long long *>(scratch + kRadixMaxPasses * kRadix + 64);  // [passes][ntiles][256]
    const size_t zero_bytes = sizeof(uint32_t) * (kRadixMaxPasses * kRadix + 64) +
                              sizeof(unsigned long long) * (size_t)passes * ntiles * kRadix;
    FMM_CUDA_TRY(cudaMemsetAsync(scratch, 0, zero_bytes, st));
    k_radix_counts<<<(unsigned)std::min<int64_t>(ceil_div(n, 256 * 8), 152 * 4), 256, 0, st>>>(keys, n, passes,
                                                                                          counts);
    FMM_LAUNCH_CHECK();
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; ++p) {
        k_radix_pass<<<(unsigned)ntiles, kSortThreads, kPassSmem, st>>>(
            ka, va, kb, vb, n, 8 * p, counts + p * kRadix, status + (int64_t)p * ntiles * kRadix, tile_counter + p,
            flags);
        FMM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        FMM_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
}

}  // namespace fmm
