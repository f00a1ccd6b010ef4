// m2l_tc.cu -- M2L translations on the 5th-generation tensor cores (tcgen05).
//
// Same regrouping as m2l.cu (targets tiled 128 at a time, one dense block per
// offset class present in the tile), computed as D = A * B^T with
//   A (128 x P2pad) = gathered source multipoles of the tile's targets,
//   B (N = P2pad x P2pad) = the class's translation matrix T(class) (rows =
//     output coefficients), both K-major,
// and D (128 x N, FP32) accumulated in tensor memory over all K-chunks of all
// classes of a work unit.  FP32 accuracy from lower-precision tensor inputs by
// the 3-term split a*b ~ ah*bh + ah*bl + al*bh with ah = hi(a), al = a - ah:
//   TF32x3: hi = a with the low 13 mantissa bits cleared, kind::tf32;
//   BF16x3: hi = bf16(a), al = bf16(a - hi), kind::f16 with BF16 inputs.
//
// The tensor core's accumulation rounds toward zero, so long accumulations in
// tensor memory drift.  Following the error-corrected split of Ootomo & Yokota
// (2022), the main products ah*bh and the correction products ah*bl + al*bh go
// to two separate accumulators.  The main one restarts at every offset-class
// block, and the blocks are summed with round-to-nearest FP32 adds into a running
// sum held in a third tensor-memory region (in the partial buffer when 3N columns
// do not fit).  The correction (about 2^-8 of the main product in BF16, 2^-11 in
// TF32) runs over all blocks of a work unit when N <= 128 and restarts with the
// main one otherwise.
//
// The class matrices B are split into hi/lo once (k_split_tables), already in
// the shared-memory layout of a stage, so a stage's B is two bulk asynchronous
// copies (cp.async.bulk, completing on an mbarrier) issued by one thread.
//
// Two kernels share this scheme.  For P2pad <= 128, k_m2l_tc_ta keeps A in
// tensor memory (described at its definition).  For larger P2pad the
// accumulators leave no tensor-memory columns for A, and k_m2l_tc stages A in
// shared memory:
//
// Roles inside a k_m2l_tc CTA (704 threads):
//   warps 0-15  producers, two groups of 8 warps that fill alternate stages:
//               gather the 128 source rows (A) of one K-chunk of 32 floats,
//               split them into hi/lo and store them in the canonical
//               no-swizzle K-major layout (8-row x 16-byte core matrices;
//               LBO = 128 B along K, SBO = 8 core matrices (TF32, 128 B rows) or
//               4 (BF16, 64 B rows) along rows).
//   warp 16     allocates tensor memory; one lane issues the MMAs and commits.
//   warps 17-20 accumulators, one per 32-lane quarter of tensor memory: after
//               each class block they read the block's main and correction
//               accumulators (two buffer pairs, alternating, when 5N columns fit)
//               and add both into the running sum.
//   warp 21     one lane issues every stage's B copies, in stage order.
// Stages are handed over through mbarriers (full: one arrival per warp of the
// stage's producer group; bfull: one arrival with the B copies' byte count;
// empty, acc_full: tcgen05.commit;
// acc_empty: one arrival per accumulator warp).  Every
// wait is bounded: on expiry the kernel raises a flag and returns after
// releasing its tensor memory.
// A work unit is (tile, range of the tile's class blocks); its 128 x N result
// goes to a partial buffer and k_m2l_reduce sums a tile's units in order.  Units
// run in the order (rank within the tile, tile): the CTAs resident at one time
// work on similar class ranges, so the class matrices they read stay in L2.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

constexpr int kProducerWarps = 8;  // per producer group
constexpr int kAccWarps = 4;
constexpr int kProducerGroups = 2;                  // they fill alternate stages
constexpr int kMmaWarp = kProducerGroups * kProducerWarps;
constexpr int kBWarp = kMmaWarp + 1 + kAccWarps;    // issues the B copies
constexpr int kThreads = (kBWarp + 1) * 32;
constexpr int kKChunk = 32;  // source floats per row per stage (128 B)
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk asynchronous copy global -> shared (16-byte aligned, size a multiple of 16),
// completing `bytes` of the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major, LBO = 128 B (next core
// matrix along K), SBO = `sbo` bytes (next 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format `fmt` (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t n)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate)
{
    if (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (store side).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
// Tensor-memory load of 16 columns without the wait: the registers are valid
// only after tmem_ld_wait() and reg_touch16() of the same array.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Keeps every use of r after the preceding wait (volatile asm statements stay in order).
__device__ __forceinline__ void reg_touch16(uint32_t (&r)[16])
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]));
}

// hi/lo split of 4 floats into one 16-byte chunk each (TF32: 4 elements).
__device__ __forceinline__ void split_tf32(float4 a, uint4 &hi, uint4 &lo)
{
    const float x[4] = {a.x, a.y, a.z, a.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t hb = __float_as_uint(x[i]) & 0xFFFFE000u;
        h[i] = hb;
        l[i] = __float_as_uint(x[i] - __uint_as_float(hb));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// hi/lo split of 8 floats into one 16-byte chunk each (BF16: 8 elements).
// BF16 keeps 8 significant bits, so hi + lo carries about 16 of the 24: the
// dropped lo*lo term and the remainder limit BF16x3 to about 1e-5 relative.
__device__ __forceinline__ void split_bf16(float4 a, float4 b, uint4 &hi, uint4 &lo)
{
    const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
        h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

struct Unit {
    int tile, e0, e1, pad;
};

// Stage layout (bytes): A_hi | A_lo | B_hi | B_lo, operand X with R rows of one
// 32-float K-chunk occupying R * RB bytes, RB = 128 (TF32) or 64 (BF16).
template <bool BF16, int N>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_tc(const Unit *__restrict__ units, const int *__restrict__ entry_class,
             const int *__restrict__ src, const float *__restrict__ M,
             const unsigned char *__restrict__ tsplit, int P2pad, int nstages,
             float *__restrict__ partial, int *__restrict__ flags, const int *__restrict__ sz)
{
    // a replayed plan launches for its unit capacity: the CTAs past the units
    // of this solve leave before touching barriers or tensor memory
    if (sz && (int)blockIdx.x >= sz[kSzUnits]) return;
    constexpr int NG = 2;                          // groups of 8 A rows per producer warp
    constexpr bool SUM_TMEM = 3 * N <= 512;        // running sum in tensor memory
    // N <= 128: [sum | main 0 | correction | main 1].  The correction
    // products (about 2^-8 of the main one) accumulate over all class blocks of
    // the unit in one buffer; the main product restarts per block in two
    // alternating buffers, so the MMAs of block b + 1 run while block b is
    // drained.  The correction sits next to both main buffers, so one MMA of
    // width 2N gives ah.bh and ah.bl together: [main 0 | corr] = ah.[bh | bl] for
    // even blocks, [corr | main 1] = ah.[bl | bh] for odd ones, whose stages hold
    // B_lo first.
    // Otherwise: [sum |] (main | correction) pairs, both restarted per block.
    constexpr bool CORR_RUN = 4 * N <= 512;
    constexpr int NBUF = CORR_RUN || 5 * N <= 512 ? 2 : 1;  // main buffers (or main/correction pairs)
    constexpr int BUF0 = SUM_TMEM ? N : 0;                   // first buffer column
    constexpr int BUFW = 2 * N;                              // columns per buffer (main 1 at 3N)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    // 32 floats of K per stage: 128 B per row in TF32, 64 B per row in BF16.
    constexpr int kstage = kKChunk;
    constexpr uint32_t RB = BF16 ? 64u : 128u;   // bytes per row per stage
    constexpr uint32_t SBO = 8u * RB;            // bytes per 8-row group
    const int nkc = (P2pad + kstage - 1) / kstage;
    const uint32_t a_bytes = 128u * RB, b_bytes = (uint32_t)N * RB;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + nstages * stage_bytes);
    uint64_t *empty = full + nstages;
    uint64_t *bfull = empty + nstages;
    uint64_t *acc_full = bfull + nstages;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *fin = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Unit U = units[blockIdx.x];
    const int nsteps = (U.e1 - U.e0) * nkc;
    constexpr int kCols = CORR_RUN ? 4 * N : BUF0 + BUFW * NBUF;  // tensor-memory columns in use
    static_assert(kCols <= 512, "tensor memory has 512 columns");
    uint32_t ncols = 32;
    while (ncols < (uint32_t)kCols) ncols <<= 1;
    const int nblocks = U.e1 - U.e0;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&full[s], kProducerWarps);  // one arrival per producer warp
            mbar_init(&bfull[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kAccWarps);  // one arrival per accumulator warp
        }
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kMmaWarp) {
        // ------------------------------------------------------------ producers
        // Group grp fills stages g = grp, grp + 2, ...  Thread (warp, lane) of the
        // group owns A rows grp8*8 + (lane & 7) for grp8 = pw + 8j (j < 2, pw = warp
        // within the group), and the 16-byte chunks (lane >> 3) + 4h of each (h < 2
        // in TF32, h = 0 in BF16).  The loads of the group's next stage are issued
        // before a stage is split and stored.
        const int grp = warp / kProducerWarps, pw = warp % kProducerWarps;
        const int sub = lane & 7, cq = lane >> 3;
        constexpr int V = 2;  // float4 per row and thread per stage
        int srow[2] = {0, 0};
        bool svalid[2] = {false, false};
        int cur_e = -1;
        auto load_stage = [&](int g, float4 (&buf)[NG][V]) {
            const int e = U.e0 + g / nkc;
            const int k0 = (g % nkc) * kstage;
            if (e != cur_e) {  // the group's first stage of a block: its source rows
                cur_e = e;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int row = (pw + 8 * j) * 8 + sub;
                    const int sidx = src[(int64_t)e * kTile + row];
                    svalid[j] = sidx >= 0;
                    srow[j] = svalid[j] ? sidx : 0;
                }
            }
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                const float *rowp = M + (int64_t)srow[j] * P2pad;
                const bool valid = svalid[j];
                if (BF16) {
                    const int kk = k0 + cq * 8;
                    buf[j][0] = valid ? *reinterpret_cast<const float4 *>(rowp + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
                    buf[j][1] = valid ? *reinterpret_cast<const float4 *>(rowp + kk + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kk = k0 + (cq + 4 * h) * 4;
                        buf[j][h] = valid ? *reinterpret_cast<const float4 *>(rowp + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        };
        // one pipeline step: consume stage g from `cur`, first issuing the loads of
        // the group's next stage into `ahead` (two register buffers in turn)
        auto step = [&](int g, float4 (&cur)[NG][V], float4 (&ahead)[NG][V]) -> bool {
            if (g + kProducerGroups < nsteps) load_stage(g + kProducerGroups, ahead);
            const int s = g % nstages;
            // the warp decides together: it synchronises before its one arrival
            const bool freed = g < nstages || mbar_wait(&empty[s], (uint32_t)((g / nstages) - 1) & 1u);
            if (!__all_sync(0xffffffffu, freed)) {
                if (lane == 0) atomicOr(&flags[kFlagTimeout], 1);
                s_abort = 1;
                return false;
            }
            if (__any_sync(0xffffffffu, s_abort != 0)) return false;
            unsigned char *st = smem + (size_t)s * stage_bytes;
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                const int row = (pw + 8 * j) * 8 + sub;
                unsigned char *dst_hi = st + (row >> 3) * SBO + (row & 7) * 16;
                unsigned char *dst_lo = dst_hi + a_bytes;
                uint4 hi, lo;
                if (BF16) {
                    split_bf16(cur[j][0], cur[j][1], hi, lo);
                    *reinterpret_cast<uint4 *>(dst_hi + cq * 128) = hi;
                    *reinterpret_cast<uint4 *>(dst_lo + cq * 128) = lo;
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        split_tf32(cur[j][h], hi, lo);
                        *reinterpret_cast<uint4 *>(dst_hi + (cq + 4 * h) * 128) = hi;
                        *reinterpret_cast<uint4 *>(dst_lo + (cq + 4 * h) * 128) = lo;
                    }
                }
            }
            fence_proxy_async();  // this thread's stores, before the tensor core reads them
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[s]);
            return true;
        };
        constexpr int D = kProducerGroups;  // stride between a group's stages
        float4 b0[NG][V], b1[NG][V];
        if (grp < nsteps) load_stage(grp, b0);
        for (int g = grp; g < nsteps; g += 2 * D) {
            if (!step(g, b0, b1)) break;
            if (g + D >= nsteps || !step(g + D, b1, b0)) break;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc(BF16 ? 1u : 2u, (uint32_t)N);
            // N <= 128: B_hi and B_lo of a stage are one 2N-row operand (same layout,
            // consecutive), and the main and correction accumulators are adjacent, so
            // one MMA of width 2N gives ah.bh and ah.bl together, reading ah once.
            constexpr bool kFuse = 2 * N <= 256;
            const uint32_t idesc2 = instr_desc(BF16 ? 1u : 2u, kFuse ? 2u * N : (uint32_t)N);
            constexpr int ksteps = (int)RB / 32;  // MMAs of 32 bytes of K per stage row
            bool ok = true;
            int g = 0;
            for (int b = 0; b < nblocks && ok; ++b) {
                const int buf = b % NBUF;
                if (b >= NBUF && !mbar_wait(&acc_empty[buf], (uint32_t)((b / NBUF) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                const uint32_t dmain = tmem + (uint32_t)(BUF0 + buf * BUFW),
                               dcorr = CORR_RUN ? tmem + (uint32_t)(2 * N) : dmain + (uint32_t)N;
                const bool odd = CORR_RUN && (b & 1);
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g % nstages;
                    if (!mbar_wait(&full[s], (uint32_t)(g / nstages) & 1u) ||
                        !mbar_wait(&bfull[s], (uint32_t)(g / nstages) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
                    const uint32_t ah = base, al = base + a_bytes, b0 = base + 2 * a_bytes,
                                   bh = odd ? b0 + b_bytes : b0, bl = odd ? b0 : b0 + b_bytes;
#pragma unroll
                    for (int k = 0; k < ksteps; ++k) {
                        const uint32_t off = (uint32_t)k * 256u;  // two core matrices along K
                        const uint32_t acc0 = (kc > 0 || k > 0) ? 1u : 0u;
                        if (CORR_RUN) {
                            if (acc0 == 0 && b > 0) {
                                // a block's first step: main restarts, the correction goes on
                                mma<BF16>(dmain, smem_desc(ah + off, SBO), smem_desc(bh + off, SBO), idesc, 0u);
                                mma<BF16>(dcorr, smem_desc(ah + off, SBO), smem_desc(bl + off, SBO), idesc, 1u);
                            } else {
                                // [main | corr] (even) or [corr | main] (odd) = ah.(B as staged)
                                mma<BF16>(odd ? dcorr : dmain, smem_desc(ah + off, SBO), smem_desc(b0 + off, SBO),
                                          idesc2, acc0);
                            }
                            mma<BF16>(dcorr, smem_desc(al + off, SBO), smem_desc(bh + off, SBO), idesc, 1u);
                        } else if (kFuse) {
                            mma<BF16>(dmain, smem_desc(ah + off, SBO), smem_desc(bh + off, SBO), idesc2, acc0);
                            mma<BF16>(dcorr, smem_desc(al + off, SBO), smem_desc(bh + off, SBO), idesc, 1u);
                        } else {
                            mma<BF16>(dcorr, smem_desc(al + off, SBO), smem_desc(bh + off, SBO), idesc, acc0);
                            mma<BF16>(dcorr, smem_desc(ah + off, SBO), smem_desc(bl + off, SBO), idesc, 1u);
                            mma<BF16>(dmain, smem_desc(ah + off, SBO), smem_desc(bh + off, SBO), idesc, acc0);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&acc_full[buf]);
            }
            if (!ok) {
                atomicOr(&flags[kFlagTimeout], 1);
                s_abort = 1;
            }
            // No MMA may still be in flight when the tensor memory is released.
            mma_commit(fin);
            if (!mbar_wait(fin, 0)) atomicOr(&flags[kFlagTimeout], 1);
        }
    } else if (warp == kBWarp) {
        if (lane == 0) {
            // ------------------------------------------------------------ B copies
            // Each stage's B (hi, lo) by two bulk copies, in stage order, as soon as the
            // stage's buffer is free.
            int issued = 0;
            for (int g = 0; g < nsteps; ++g) {
                const int s = g % nstages;
                if (g >= nstages && !mbar_wait(&empty[s], (uint32_t)((g / nstages) - 1) & 1u)) {
                    atomicOr(&flags[kFlagTimeout], 1);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                unsigned char *st = smem + (size_t)s * stage_bytes;
                const int e = U.e0 + g / nkc, kc = g % nkc;
                const unsigned char *bsrc = tsplit + ((int64_t)entry_class[e] * nkc + kc) * 2 * (int64_t)b_bytes;
                const bool lo_first = CORR_RUN && ((g / nkc) & 1);  // odd blocks: [B_lo | B_hi]
                mbar_arrive_expect_tx(&bfull[s], 2 * b_bytes);
                bulk_g2s(st + 2 * a_bytes + (lo_first ? b_bytes : 0), bsrc, b_bytes, &bfull[s]);
                bulk_g2s(st + 2 * a_bytes + (lo_first ? 0 : b_bytes), bsrc + b_bytes, b_bytes, &bfull[s]);
                issued = g + 1;
            }
            // no B copy may still be landing when the CTA ends (matters after an abort)
            for (int g = issued - 1; g >= 0 && g >= issued - nstages; --g)
                if (!mbar_wait(&bfull[g % nstages], (uint32_t)(g / nstages) & 1u)) atomicOr(&flags[kFlagTimeout], 1);
        }
    } else {
        // ------------------------------------------------------------ accumulators
        // (warps 17-20: warp & 3 covers the four lane quarters)
        // sum_b = sum_{b-1} + (main_b + corr_b), FP32 round-to-nearest, per element;
        // with the running correction: sum_b = sum_{b-1} + main_b, and the
        // correction is added once after the last block.
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        float *out = partial + ((int64_t)blockIdx.x * 128 + row) * P2pad;
        for (int b = 0; b < nblocks; ++b) {
            const int buf = b % NBUF;
            // The warp leaves together: the tensor-memory loads below are warp-wide.
            if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(b / NBUF) & 1u))) {
                atomicOr(&flags[kFlagTimeout], 1);
                break;
            }
            tc_fence_after();
            const uint32_t dmain = tmem + lane_off + (uint32_t)(BUF0 + buf * BUFW);
            const uint32_t dcorr = CORR_RUN ? tmem + lane_off + (uint32_t)(2 * N) : dmain + (uint32_t)N;
            const bool last = b + 1 == nblocks;
            if (CORR_RUN) {
                // sum_b = sum_{b-1} + main_b in tensor memory; after the last block the
                // correction is loaded on its own, which keeps two chunks in registers
                const uint32_t dsum = tmem + lane_off;
                for (int c0 = 0; c0 < N; c0 += 16) {
                    uint32_t rm[16], rs[16];
                    tmem_ld16_issue(dmain + (uint32_t)c0, rm);
                    if (b > 0) tmem_ld16_issue(dsum + (uint32_t)c0, rs);
                    tmem_ld_wait();
                    reg_touch16(rm);
                    if (b > 0) reg_touch16(rs);
                    float vs[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        vs[i] = b > 0 ? __uint_as_float(rs[i]) + __uint_as_float(rm[i]) : __uint_as_float(rm[i]);
                    if (last) {
                        uint32_t rc[16];
                        tmem_ld16_issue(dcorr + (uint32_t)c0, rc);
                        tmem_ld_wait();
                        reg_touch16(rc);
#pragma unroll
                        for (int i = 0; i < 16; ++i) vs[i] += __uint_as_float(rc[i]);
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4 *>(out + c0 + i) = make_float4(vs[i], vs[i + 1], vs[i + 2], vs[i + 3]);
                    } else {
                        tmem_st16(dsum + (uint32_t)c0, vs);
                    }
                }
            }
            for (int c0 = 0; c0 < (CORR_RUN ? 0 : N); c0 += 16) {
                float vm[16], vc[16], vs[16];
                {
                    // the chunk's main, correction and running-sum columns under one wait
                    uint32_t rm[16], rc[16], rs[16];
                    const bool lds = SUM_TMEM && b > 0;
                    tmem_ld16_issue(dmain + (uint32_t)c0, rm);
                    tmem_ld16_issue(dcorr + (uint32_t)c0, rc);
                    if (lds) tmem_ld16_issue(tmem + lane_off + (uint32_t)c0, rs);
                    tmem_ld_wait();
                    reg_touch16(rm);
                    reg_touch16(rc);
                    if (lds) reg_touch16(rs);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        vm[i] = __uint_as_float(rm[i]);
                        vc[i] = __uint_as_float(rc[i]);
                        vs[i] = lds ? __uint_as_float(rs[i]) : 0.f;
                    }
                }
                if (b > 0) {
                    if (!SUM_TMEM) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            const float4 t = *reinterpret_cast<const float4 *>(out + c0 + i);
                            vs[i] = t.x, vs[i + 1] = t.y, vs[i + 2] = t.z, vs[i + 3] = t.w;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) vs[i] += vm[i] + vc[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) vs[i] = vm[i] + vc[i];
                }
                if (last || !SUM_TMEM) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4 *>(out + c0 + i) = make_float4(vs[i], vs[i + 1], vs[i + 2], vs[i + 3]);
                } else {
                    tmem_st16(tmem + lane_off + (uint32_t)c0, vs);
                }
            }
            if (SUM_TMEM && !last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// A operand in tensor memory (N = P2pad <= 128).
//
// The same products, accumulators and order of additions as k_m2l_tc, with the
// gathered source rows held in tensor memory instead of shared memory: the
// producers split each row into hi/lo in registers and write both with
// tcgen05.st, and the MMAs take A from tensor memory (tcgen05.mma's [a-tmem]
// form).  Shared memory then carries only the class matrices: their bulk copies
// and the MMAs' reads of B.  Per stage of 32 K values (TF32, N = 128) that is
// 32 KB written and 48 KB read, against 32 + 32 KB written and 80 KB read with A
// in shared memory, where shared memory, not the tensor pipe, set the pace.
//
// Tensor-memory columns: [main 0 | correction | main 1] at 0, N, 2N (as in
// k_m2l_tc with the running correction), and a ring of A stages at 384..511:
// TF32 stages of 64 columns (hi 32 K values, lo 32), BF16 stages of 32 (two
// values per 32-bit column).  Row r of A is tensor-memory lane r.
//
// Roles (576 threads):
//   warps 0-7   producers, two per 32-lane quarter (warp & 3): thread (warp,
//               lane) owns A row 32 (warp & 3) + lane and half (warp >> 2) of
//               each stage's 32 K values; loads run two stages ahead.
//   warp 8      allocates tensor memory; one lane issues the MMAs and commits.
//   warps 9-16  accumulators, two per lane quarter, each owning half of the N
//               columns of its 32 rows: the running sum of the class blocks'
//               main products is kept in registers (FP32 round-to-nearest adds,
//               the same order as k_m2l_tc), the correction added after the last
//               block.
//   warp 17     one lane issues every stage's B copies, in stage order.
namespace ta {
constexpr int kProducers = 8;
constexpr int kMmaWarp = 8;
constexpr int kAcc0 = 9, kAccWarps = 8;
constexpr int kBWarp = kAcc0 + kAccWarps;
constexpr int kThreads = (kBWarp + 1) * 32;
constexpr uint32_t kACol = 384;  // first tensor-memory column of the A ring
constexpr int kTmemCols = 512;
}  // namespace ta

// Tensor-memory store of 8 consecutive 32-bit columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (tensor memory) (+)= A (tensor memory, lane = row) * B (shared memory)^T.
template <bool BF16>
__device__ __forceinline__ void mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate)
{
    if (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
    }
}

template <bool BF16, int N>
__global__ void __launch_bounds__(ta::kThreads, 1)
    k_m2l_tc_ta(const Unit *__restrict__ units, const int *__restrict__ entry_class,
                const int *__restrict__ src, const float *__restrict__ M,
                const unsigned char *__restrict__ tsplit, int nbstages,
                float *__restrict__ partial, int *__restrict__ flags, const int *__restrict__ sz)
{
    static_assert(N % 32 == 0 && N <= 128, "N = P2pad <= 128, a multiple of 32");
    if (sz && (int)blockIdx.x >= sz[kSzUnits]) return;
    constexpr int P2pad = N;
    constexpr int ACOLS = BF16 ? 32 : 64;      // tensor-memory columns per A stage (hi + lo)
    constexpr int NAST = 128 / ACOLS;          // A stages in the ring
    constexpr int KSTEPS = ACOLS / 16;         // MMAs (8 columns of A each) per stage
    constexpr uint32_t RB = BF16 ? 64u : 128u;  // bytes per B row per stage
    constexpr uint32_t SBO = 8u * RB;
    constexpr uint32_t b_bytes = (uint32_t)N * RB;
    constexpr int nkc = P2pad / kKChunk;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    uint64_t *bfull = reinterpret_cast<uint64_t *>(smem + (size_t)nbstages * 2 * b_bytes);
    uint64_t *bempty = bfull + nbstages;
    uint64_t *afull = bempty + nbstages;
    uint64_t *aempty = afull + NAST;
    uint64_t *acc_full = aempty + NAST;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *fin = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Unit U = units[blockIdx.x];
    const int nblocks = U.e1 - U.e0;
    const int nsteps = nblocks * nkc;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < nbstages; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (int s = 0; s < NAST; ++s) {
            mbar_init(&afull[s], ta::kProducers);  // one arrival per producer warp
            mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], ta::kAccWarps);
        }
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == ta::kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"((uint32_t)ta::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < ta::kProducers) {
        // ------------------------------------------------------------ producers
        const int quad = warp & 3, half = warp >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        // the row's source index of the next block is read one block ahead, so a
        // block's first rows wait for one load, not two in a chain
        int cur_e = -1, srow = 0, next_src = nblocks > 0 ? src[(int64_t)U.e0 * kTile + row] : -1;
        bool svalid = false;
        auto load = [&](int g, float4 (&buf)[4]) {
            const int e = U.e0 + g / nkc;
            if (e != cur_e) {  // a block's first stage: the row's source
                cur_e = e;
                svalid = next_src >= 0;
                srow = svalid ? next_src : 0;
                if (e + 1 < U.e1) next_src = src[(int64_t)(e + 1) * kTile + row];
            }
            const float4 *p = reinterpret_cast<const float4 *>(M + (int64_t)srow * P2pad + (g % nkc) * kKChunk +
                                                               half * 16);
#pragma unroll
            for (int v = 0; v < 4; ++v) buf[v] = svalid ? p[v] : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto fill = [&](int g, const float4 (&buf)[4]) -> bool {
            const int s = g % NAST;
            const bool freed = g < NAST || mbar_wait(&aempty[s], (uint32_t)((g / NAST) - 1) & 1u);
            if (!__all_sync(0xffffffffu, freed)) {
                if (lane == 0) atomicOr(&flags[kFlagTimeout], 1);
                s_abort = 1;
                return false;
            }
            if (__any_sync(0xffffffffu, s_abort != 0)) return false;
            tc_fence_after();
            const uint32_t col = tmem + lane_off + ta::kACol + (uint32_t)(s * ACOLS);
            if (BF16) {
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int v = 0; v < 4; v += 2) {
                    uint4 h, l;
                    split_bf16(buf[v], buf[v + 1], h, l);
                    hi[2 * v] = h.x, hi[2 * v + 1] = h.y, hi[2 * v + 2] = h.z, hi[2 * v + 3] = h.w;
                    lo[2 * v] = l.x, lo[2 * v + 1] = l.y, lo[2 * v + 2] = l.z, lo[2 * v + 3] = l.w;
                }
                tmem_st8u(col + (uint32_t)(half * 8), hi);
                tmem_st8u(col + (uint32_t)(ACOLS / 2 + half * 8), lo);
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q) {  // 8 K values at a time
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        uint4 h, l;
                        split_tf32(buf[2 * q + v], h, l);
                        hi[4 * v] = h.x, hi[4 * v + 1] = h.y, hi[4 * v + 2] = h.z, hi[4 * v + 3] = h.w;
                        lo[4 * v] = l.x, lo[4 * v + 1] = l.y, lo[4 * v + 2] = l.z, lo[4 * v + 3] = l.w;
                    }
                    tmem_st8u(col + (uint32_t)(half * 16 + q * 8), hi);
                    tmem_st8u(col + (uint32_t)(ACOLS / 2 + half * 16 + q * 8), lo);
                }
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[s]);
            return true;
        };
        // loads run two stages ahead of the stage being written (three buffers in turn)
        float4 r0[4], r1[4], r2[4];
        if (0 < nsteps) load(0, r0);
        if (1 < nsteps) load(1, r1);
        for (int g = 0; g < nsteps; g += 3) {
            if (g + 2 < nsteps) load(g + 2, r2);
            if (!fill(g, r0) || g + 1 >= nsteps) break;
            if (g + 3 < nsteps) load(g + 3, r0);
            if (!fill(g + 1, r1) || g + 2 >= nsteps) break;
            if (g + 4 < nsteps) load(g + 4, r1);
            if (!fill(g + 2, r2)) break;
        }
    } else if (warp == ta::kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc(BF16 ? 1u : 2u, (uint32_t)N);
            const uint32_t idesc2 = instr_desc(BF16 ? 1u : 2u, 2u * N);
            bool ok = true;
            int g = 0;
            for (int b = 0; b < nblocks && ok; ++b) {
                const int buf = b & 1;
                if (b >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((b >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dmain = tmem + (uint32_t)(buf ? 2 * N : 0), dcorr = tmem + (uint32_t)N;
                const bool odd = b & 1;
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int sa = g % NAST, sb = g % nbstages;
                    if (!mbar_wait(&afull[sa], (uint32_t)(g / NAST) & 1u) ||
                        !mbar_wait(&bfull[sb], (uint32_t)(g / nbstages) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ah = tmem + ta::kACol + (uint32_t)(sa * ACOLS), al = ah + (uint32_t)(ACOLS / 2);
                    const uint32_t b0 = smem_u32(smem + (size_t)sb * 2 * b_bytes);
                    const uint32_t bh = odd ? b0 + b_bytes : b0, bl = odd ? b0 : b0 + b_bytes;
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k) {
                        const uint32_t ka = (uint32_t)k * 8u;    // 8 columns of A
                        const uint32_t kb = (uint32_t)k * 256u;  // two core matrices of B along K
                        const uint32_t acc0 = (kc > 0 || k > 0) ? 1u : 0u;
                        if (acc0 == 0 && b > 0) {
                            // a block's first step: main restarts, the correction goes on
                            mma_ta<BF16>(dmain, ah + ka, smem_desc(bh + kb, SBO), idesc, 0u);
                            mma_ta<BF16>(dcorr, ah + ka, smem_desc(bl + kb, SBO), idesc, 1u);
                        } else {
                            // [main 0 | corr] (even) or [corr | main 1] (odd) = ah.(B as staged)
                            mma_ta<BF16>(odd ? dcorr : dmain, ah + ka, smem_desc(b0 + kb, SBO), idesc2, acc0);
                        }
                        mma_ta<BF16>(dcorr, al + ka, smem_desc(bh + kb, SBO), idesc, 1u);
                    }
                    mma_commit(&aempty[sa]);
                    mma_commit(&bempty[sb]);
                }
                if (ok) mma_commit(&acc_full[buf]);
            }
            if (!ok) {
                atomicOr(&flags[kFlagTimeout], 1);
                s_abort = 1;
            }
            mma_commit(fin);
            if (!mbar_wait(fin, 0)) atomicOr(&flags[kFlagTimeout], 1);
        }
    } else if (warp == ta::kBWarp) {
        // ------------------------------------------------------------ B copies
        if (lane == 0) {
            int issued = 0;
            for (int g = 0; g < nsteps; ++g) {
                const int s = g % nbstages;
                if (g >= nbstages && !mbar_wait(&bempty[s], (uint32_t)((g / nbstages) - 1) & 1u)) {
                    atomicOr(&flags[kFlagTimeout], 1);
                    s_abort = 1;
                    break;
                }
                if (s_abort) break;
                unsigned char *st = smem + (size_t)s * 2 * b_bytes;
                const int e = U.e0 + g / nkc, kc = g % nkc;
                const unsigned char *bsrc = tsplit + ((int64_t)entry_class[e] * nkc + kc) * 2 * (int64_t)b_bytes;
                const bool lo_first = (g / nkc) & 1;  // odd blocks: [B_lo | B_hi]
                mbar_arrive_expect_tx(&bfull[s], 2 * b_bytes);
                bulk_g2s(st + (lo_first ? b_bytes : 0), bsrc, b_bytes, &bfull[s]);
                bulk_g2s(st + (lo_first ? 0 : b_bytes), bsrc + b_bytes, b_bytes, &bfull[s]);
                issued = g + 1;
            }
            for (int g = issued - 1; g >= 0 && g >= issued - nbstages; --g)
                if (!mbar_wait(&bfull[g % nbstages], (uint32_t)(g / nbstages) & 1u))
                    atomicOr(&flags[kFlagTimeout], 1);
        }
    } else {
        // ------------------------------------------------------------ accumulators
        // sum_b = sum_{b-1} + main_b (FP32 round-to-nearest, per element); after
        // the last block, + correction.
        constexpr int NH = N / 2;
        const int quad = warp & 3, half = (warp - ta::kAcc0) >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        const uint32_t c0 = (uint32_t)(half * NH);
        float sum[NH];
        bool done = true;
        for (int b = 0; b < nblocks; ++b) {
            const int buf = b & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(b >> 1) & 1u))) {
                atomicOr(&flags[kFlagTimeout], 1);
                done = false;
                break;
            }
            tc_fence_after();
            const uint32_t dmain = tmem + lane_off + (uint32_t)(buf ? 2 * N : 0) + c0;
#pragma unroll
            for (int c = 0; c < NH; c += 16) {
                uint32_t r[16];
                tmem_ld16_issue(dmain + (uint32_t)c, r);
                tmem_ld_wait();
                reg_touch16(r);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[c + i] = b > 0 ? sum[c + i] + __uint_as_float(r[i]) : __uint_as_float(r[i]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        if (done && nblocks > 0) {
            float *out = partial + ((int64_t)blockIdx.x * 128 + row) * P2pad + c0;
#pragma unroll
            for (int c = 0; c < NH; c += 16) {
                uint32_t r[16];
                tmem_ld16_issue(tmem + lane_off + (uint32_t)N + c0 + (uint32_t)c, r);
                tmem_ld_wait();
                reg_touch16(r);
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4 *>(out + c + i) =
                        make_float4(sum[c + i] + __uint_as_float(r[i]), sum[c + i + 1] + __uint_as_float(r[i + 1]),
                                    sum[c + i + 2] + __uint_as_float(r[i + 2]),
                                    sum[c + i + 3] + __uint_as_float(r[i + 3]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == ta::kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)ta::kTmemCols)
                     : "memory");
    }
}

// L rows of a tile = sum of its units' partials, in the order tile_units lists
// them (the tile's class order).
__global__ void k_m2l_reduce(const int *__restrict__ unit_base, const int *__restrict__ tile_units,
                             const float *__restrict__ partial, const int *__restrict__ tile_cells, int P2pad,
                             float *__restrict__ L)
{
    const int tile = blockIdx.x;
    const int u0 = unit_base[tile], u1 = unit_base[tile + 1];
    const int nq = P2pad / 4;
    for (int i = threadIdx.x; i < kTile * nq; i += blockDim.x) {
        const int row = i / nq, q4 = i % nq;
        const int cell = tile_cells[(int64_t)tile * kTile + row];
        if (cell < 0) continue;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = u0; i < u1; ++i) {
            const int u = tile_units[i];
            const float4 v = reinterpret_cast<const float4 *>(partial + ((int64_t)u * 128 + row) * P2pad)[q4];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
        }
        reinterpret_cast<float4 *>(L + (int64_t)cell * P2pad)[q4] = a;
    }
}

// Class matrices T (FP32 [slot][P2pad][P2pad]) split into hi/lo in the stage
// layout: for slot, K-chunk kc (32 floats): N rows x RB bytes of hi, then of lo,
// row r's 16-byte chunk c at (r >> 3) * 8 RB + (r & 7) * 16 + c * 128.
// One thread per (slot, kc, row, chunk).
template <bool BF16>
__global__ void k_split_tables(const float *__restrict__ table, int slot0, int nslots, int P2pad,
                               unsigned char *__restrict__ out)
{
    constexpr int RB = BF16 ? 64 : 128, CH = RB / 16, EPC = BF16 ? 8 : 4;  // elements per chunk
    const int N = P2pad, nkc = P2pad / kKChunk;
    const int64_t per_slot = (int64_t)nkc * N * CH;
    const int64_t total = per_slot * nslots;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int slot = slot0 + (int)(i / per_slot);
        int64_t rem = i % per_slot;
        const int kc = (int)(rem / (N * CH));
        rem %= N * CH;
        const int r = (int)(rem / CH), ch = (int)(rem % CH);
        const float *src = table + ((int64_t)slot * P2pad + r) * P2pad + kc * kKChunk + ch * EPC;
        const float4 a = *reinterpret_cast<const float4 *>(src);
        uint4 hi, lo;
        if (BF16)
            split_bf16(a, *reinterpret_cast<const float4 *>(src + 4), hi, lo);
        else
            split_tf32(a, hi, lo);
        const int64_t bbytes = (int64_t)N * RB;
        unsigned char *base = out + ((int64_t)slot * nkc + kc) * 2 * bbytes + (r >> 3) * 8 * RB + (r & 7) * 16 + ch * 128;
        *reinterpret_cast<uint4 *>(base) = hi;
        *reinterpret_cast<uint4 *>(base + bbytes) = lo;
    }
}

// Failure-detection self-test: an mbarrier that nothing arrives at, waited on
// with the same bounded loop as the M2L pipeline (polls limit), so the wait must
// give up, raise the timeout flag and return.
__global__ void k_wait_selftest(uint32_t polls, int *__restrict__ flags)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(&bar);
        bool done = false;
        for (uint32_t it = 0; it < polls && !done; ++it) {
            uint32_t d;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(d)
                : "r"(a), "r"(0u)
                : "memory");
            done = d != 0;
        }
        if (!done) atomicOr(&flags[kFlagTimeout], 1);
    }
}

}  // namespace

bool m2l_tc_supported(int P2pad) { return P2pad <= 256; }

void launch_wait_selftest(uint32_t polls, int *flags, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(polls, flags);
    FMM_LAUNCH_CHECK();
}

size_t m2l_split_bytes(int P2pad, bool bf16, int nslots)
{
    return (size_t)nslots * (P2pad / kKChunk) * 2 * (size_t)P2pad * (bf16 ? 64 : 128);
}

void launch_split_tables(bool bf16, const float *table, int slot0, int nslots, int P2pad, unsigned char *out,
                         cudaStream_t st)
{
    if (nslots <= 0) return;
    const int64_t total = (int64_t)nslots * (P2pad / kKChunk) * P2pad * (bf16 ? 4 : 8);
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16);
    if (bf16)
        k_split_tables<true><<<grid, 256, 0, st>>>(table, slot0, nslots, P2pad, out);
    else
        k_split_tables<false><<<grid, 256, 0, st>>>(table, slot0, nslots, P2pad, out);
    FMM_LAUNCH_CHECK();
}

size_t m2l_tc_smem(int P2pad, bool bf16, int &nstages)
{
    const size_t rb = bf16 ? 64 : 128;
    const size_t stage = 2 * 128 * rb + 2 * (size_t)P2pad * rb;
    nstages = (int)std::min<size_t>(bf16 ? 6 : 4, (200 * 1024) / stage);
    if (nstages < 2) nstages = 2;
    return nstages * stage + 1024 /*alignment*/ + (3 * nstages + 5) * 8 + 16;
}

// Shared memory of k_m2l_tc_ta: a ring of B stages (hi and lo of N rows of 32 K
// values), its barriers and the 1024-byte alignment slack.
static size_t m2l_tc_ta_smem(int P2pad, bool bf16, int &nbstages)
{
    const size_t stage = 2 * (size_t)P2pad * (bf16 ? 64 : 128);
    nbstages = (int)std::min<size_t>(4, (192 * 1024) / stage);  // more stages measured slower (L1 share)
    return nbstages * stage + 1024 + (2 * nbstages + 2 * 4 + 5) * 8 + 16;
}

void launch_m2l_tc(bool bf16, int nunits, const void *units, int ntiles, const int *unit_base,
                   const int *tile_units, const int *entry_class, const int *src, const int *tile_cells,
                   const float *M, const unsigned char *tsplit, int P2pad, float *partial, float *L,
                   int *flags, cudaStream_t st, const int *sz)
{
    if (nunits > 0 && P2pad <= 128) {
        int nb = 0;
        const size_t smem = m2l_tc_ta_smem(P2pad, bf16, nb);
#define FMM_M2L_TA_LAUNCH(B, NN)                                                                     \
    do {                                                                                            \
        set_smem_limit_once((const void *)k_m2l_tc_ta<B, NN>, (int)smem);                           \
        k_m2l_tc_ta<B, NN><<<nunits, ta::kThreads, smem, st>>>(static_cast<const Unit *>(units), entry_class, \
                                                               src, M, tsplit, nb, partial, flags, sz); \
    } while (0)
#define FMM_M2L_TA_BY_N(B)                              \
    do {                                                \
        switch (P2pad) {                                \
            case 32: FMM_M2L_TA_LAUNCH(B, 32); break;   \
            case 64: FMM_M2L_TA_LAUNCH(B, 64); break;   \
            case 96: FMM_M2L_TA_LAUNCH(B, 96); break;   \
            default: FMM_M2L_TA_LAUNCH(B, 128); break;  \
        }                                               \
    } while (0)
        if (bf16)
            FMM_M2L_TA_BY_N(true);
        else
            FMM_M2L_TA_BY_N(false);
#undef FMM_M2L_TA_BY_N
#undef FMM_M2L_TA_LAUNCH
        FMM_LAUNCH_CHECK();
        nunits = 0;  // done: only the reduction below remains
    }
    int nstages = 0;
    const size_t smem = m2l_tc_smem(P2pad, bf16, nstages);
    if (nunits > 0) {
#define FMM_M2L_TC_LAUNCH(B, NN)                                                                    \
    do {                                                                                           \
        set_smem_limit_once((const void *)k_m2l_tc<B, NN>, (int)smem);                              \
        k_m2l_tc<B, NN><<<nunits, kThreads, smem, st>>>(static_cast<const Unit *>(units), entry_class, \
                                                        src, M, tsplit, P2pad, nstages, partial, flags, sz); \
    } while (0)
#define FMM_M2L_TC_BY_N(B)                                  \
    do {                                                    \
        switch (P2pad) {                                    \
            case 32: FMM_M2L_TC_LAUNCH(B, 32); break;       \
            case 64: FMM_M2L_TC_LAUNCH(B, 64); break;       \
            case 96: FMM_M2L_TC_LAUNCH(B, 96); break;       \
            case 128: FMM_M2L_TC_LAUNCH(B, 128); break;     \
            case 160: FMM_M2L_TC_LAUNCH(B, 160); break;     \
            case 192: FMM_M2L_TC_LAUNCH(B, 192); break;     \
            case 224: FMM_M2L_TC_LAUNCH(B, 224); break;     \
            default: FMM_M2L_TC_LAUNCH(B, 256); break;      \
        }                                                   \
    } while (0)
        if (bf16)
            FMM_M2L_TC_BY_N(true);
        else
            FMM_M2L_TC_BY_N(false);
#undef FMM_M2L_TC_BY_N
#undef FMM_M2L_TC_LAUNCH
        FMM_LAUNCH_CHECK();
    }
    k_m2l_reduce<<<ntiles, 256, 0, st>>>(unit_base, tile_units, partial, tile_cells, P2pad, L);
    FMM_LAUNCH_CHECK();
}


// Work units of a replayed plan, built as the host builds them for a solve: tile
// t has ceil(blocks_t / chunk) units, unit r of tile t covers its blocks
// [eb_t + r chunk, min(eb_t + (r + 1) chunk, eb_{t+1})).  The units of chunk
// blocks run first in the order (r, t), then each tile's shorter last unit,
// longer ones first (kUnitBuckets size classes, tile order within one): the
// units are one CTA each and an SM takes the next as it frees, so short units
// last even out the SMs' ends (longest-first list scheduling).  One block: per
// rank r, then per size class, a block-wide scan over the tiles gives each unit
// its place.
__global__ void __launch_bounds__(1024)
    k_build_units(const int *__restrict__ entry_base, int ntiles_cap, int chunk, int units_cap,
                  M2LUnit *__restrict__ units, int *__restrict__ unit_base, int *__restrict__ tile_units,
                  int *__restrict__ sz)
{
    __shared__ int s_part[32];
    __shared__ int s_total, s_maxr;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int per = (ntiles_cap + nthr - 1) / nthr;  // tiles per thread, contiguous
    const int t0 = min(ntiles_cap, tid * per), t1 = min(ntiles_cap, t0 + per);
    auto nut = [&](int t) { return (entry_base[t + 1] - entry_base[t] + chunk - 1) / chunk; };
    // block-wide exclusive scan of one value per thread (in thread order)
    auto scan = [&](int v, int &total) {
        const int lane = tid & 31, w = tid >> 5;
        int x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        __syncthreads();
        if (lane == 31) s_part[w] = x;
        __syncthreads();
        if (w == 0) {
            const int nw = (nthr + 31) >> 5;
            int y = lane < nw ? s_part[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const int z = __shfl_up_sync(0xffffffffu, y, d);
                if (lane >= d) y += z;
            }
            if (lane < nw) s_part[lane] = y;  // inclusive per warp
            if (lane == 31) s_total = y;
        }
        __syncthreads();
        total = s_total;
        return x - v + (w > 0 ? s_part[w - 1] : 0);
    };
    // unit_base: exclusive scan of the units per tile
    int mine = 0, maxr = 0;
    for (int t = t0; t < t1; ++t) {
        const int u = nut(t);
        mine += u;
        maxr = max(maxr, u);
    }
    if (tid == 0) s_maxr = 0;
    __syncthreads();
    atomicMax(&s_maxr, maxr);
    int nunits = 0;
    int base = scan(mine, nunits);
    const bool fits = nunits <= units_cap;
    for (int t = t0; t < t1; ++t) {
        unit_base[t] = fits ? base : 0;
        base += fits ? nut(t) : 0;
    }
    if (tid == nthr - 1) unit_base[ntiles_cap] = fits ? nunits : 0;
    if (tid == 0) {
        sz[kSzUnits] = fits ? nunits : 0;
        if (!fits) sz[kSzAbort] = 1;
    }
    if (!fits) return;
    __syncthreads();
    const int R = s_maxr;
    // size class of a unit: kUnitBuckets for a full one, else its size's class
    auto bucket = [&](int t, int r) {
        const int e0 = entry_base[t] + r * chunk;
        const int n = min(chunk, entry_base[t + 1] - e0);
        return n == chunk ? kUnitBuckets : n * kUnitBuckets / (chunk + 1);
    };
    auto place = [&](int t, int r, int &pos) {
        const int e0 = entry_base[t] + r * chunk;
        units[pos] = {t, e0, min(e0 + chunk, entry_base[t + 1]), 0};
        tile_units[unit_base[t] + r] = pos;
        ++pos;
    };
    int done = 0;  // units placed so far
    for (int r = 0; r < R; ++r) {  // full units, rank by rank
        int cnt = 0;
        for (int t = t0; t < t1; ++t) cnt += nut(t) > r && bucket(t, r) == kUnitBuckets;
        int total = 0;
        int pos = done + scan(cnt, total);
        for (int t = t0; t < t1; ++t)
            if (nut(t) > r && bucket(t, r) == kUnitBuckets) place(t, r, pos);
        done += total;
    }
    for (int k = kUnitBuckets - 1; k >= 0; --k) {  // each tile's shorter last unit
        int cnt = 0;
        for (int t = t0; t < t1; ++t) cnt += nut(t) > 0 && bucket(t, nut(t) - 1) == k;
        int total = 0;
        int pos = done + scan(cnt, total);
        for (int t = t0; t < t1; ++t)
            if (nut(t) > 0 && bucket(t, nut(t) - 1) == k) place(t, nut(t) - 1, pos);
        done += total;
    }
}

}  // namespace fmm
