// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both are building blocks of the tree construction (sorting Morton keys, the
// paper's tree build which it ran on the host CPU) and of the list compaction
// in the dual tree traversal.  Written for coalesced HBM access: each block
// owns a contiguous tile, and the radix scatter reorders a whole tile in shared
// memory first so that each digit's run is written contiguously.
#include "common.cuh"

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

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kRadix = 256;

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             uint32_t *__restrict__ hist, int ntiles)
{
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    // digit-major layout: all tiles of digit 0, then digit 1, ...
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: ranks keys within the tile (index order), reorders
// the tile in shared memory by digit, then writes each digit run contiguously.
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                    const uint32_t *__restrict__ offs, int ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);                 // kSortTile keys
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);           // kSortTile vals
    uint32_t *wcnt = sv + kSortTile;                                       // [8 warps][256]
    uint32_t *run = wcnt + 8 * kRadix;                                     // [256] running count
    uint32_t *tile_off = run + kRadix;                                     // [256]
    uint32_t *gbase = tile_off + kRadix;                                   // [256]
    uint32_t *sw = gbase + kRadix;                                         // [33] scan scratch

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int tile_n = (int)(n - base < (int64_t)kSortTile ? n - base : (int64_t)kSortTile);
    run[tid] = 0;
    gbase[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;

    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = i * kSortThreads + tid;
        const bool valid = li < tile_n;
        key[i] = valid ? kin[base + li] : ~0ull;
        val[i] = valid ? vin[base + li] : 0u;
    }
    for (int i = 0; i < kSortItems; ++i) {
        for (int d = tid; d < 8 * kRadix; d += kSortThreads) wcnt[d] = 0;
        __syncthreads();
        const int li = i * kSortThreads + tid;
        const bool valid = li < tile_n;
        const uint32_t dig = (uint32_t)(key[i] >> shift) & 0xffu;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        unsigned peers = __match_any_sync(0xffffffffu, valid ? dig : 0x100u);
        peers &= active;
        uint32_t lr = __popc(peers & lt_mask);
        if (valid && lr == 0) wcnt[warp * kRadix + dig] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over the 8 warps, then add the running count
        {
            const int d = tid;
            uint32_t acc = run[d];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                uint32_t c = wcnt[w * kRadix + d];
                wcnt[w * kRadix + d] = acc;
                acc += c;
            }
            run[d] = acc;
        }
        __syncthreads();
        rank[i] = valid ? wcnt[warp * kRadix + dig] + lr : 0u;
        __syncthreads();
    }
    // tile-level digit offsets (exclusive scan of run[] over digits)
    {
        uint32_t tot;
        uint32_t ex = block_exclusive<uint32_t>(run[tid], sw, &tot);
        tile_off[tid] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int li = i * kSortThreads + tid;
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
        const uint32_t dst = gbase[dig] + (li - tile_off[dig]);
        kout[dst] = k;
        vout[dst] = sv[li];
    }
}

constexpr size_t kScatterSmem = (size_t)kSortTile * 8 + (size_t)kSortTile * 4 +
                                (8 * kRadix + 3 * kRadix + 33) * 4;

}  // namespace

int64_t radix_hist_elems(int64_t n) { return (int64_t)kRadix * ceil_div(n, kSortTile) + 1; }

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st)
{
    if (n <= 1) return;
    set_smem_limit_once((const void *)k_radix_scatter, (int)kScatterSmem);
    const int ntiles = (int)ceil_div(n, kSortTile);
    const int64_t nh = (int64_t)kRadix * ntiles;
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, shift, hist, ntiles);
        FMM_LAUNCH_CHECK();
        scan_exclusive<uint32_t>(hist, hist, nh, nullptr, scan_tmp, st);
        k_radix_scatter<<<ntiles, kSortThreads, kScatterSmem, st>>>(ka, va, kb, vb, n, shift,
                                                                    hist, ntiles);
        FMM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
        ++passes;
    }
    if (passes & 1) {
        FMM_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
}

}  // namespace fmm
