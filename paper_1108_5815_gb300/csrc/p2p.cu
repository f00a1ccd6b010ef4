// p2p.cu -- particle-particle near field, the all-pairs direct sum, and the
// final combination of near and far fields in the caller's order.
//
// P2P (the paper's "local evaluation", which dominates its GPU run time,
// Fig. "breakdown") sums q_j / r and q_j (x_j - x_i) / r^3 over the sources of
// the target leaf's P2P list.  Target-parallel (one lane per target particle,
// the layout of Nyland et al. that the paper recounts): no reduction across
// threads, source tiles staged through shared memory and broadcast.
//
// Per interaction: 3 FADD for the offset, 3 for r^2, one MUFU rsqrt with one
// Newton step y <- y (3/2 - r^2 y^2 / 2), then phi += q y and
// grad += q y^3 d.  Pairs at r = 0 (the particle itself, coincident points)
// contribute nothing: rsqrt(0) = inf makes the Newton step NaN and
// max(NaN, 0) = 0 removes it without a branch.
// Each lane takes its target against two sources at a time with the packed
// FP32x2 instructions (add/sub/mul/fma.rn.f32x2): one instruction does the same
// operation for both sources, which halves the issue slots of the arithmetic;
// only the rsqrt and the NaN guard stay scalar.  Sources are staged in shared
// memory as four arrays (x, y, z, q), so a pair of consecutive sources is one
// 64-bit load per component.
#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two packed FP32 values (first in the low half).
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct Target2 {
    f2 x, y, z;          // the target's coordinates in both halves
    f2 mhalf, threehalf; // (-1/2, -1/2), (3/2, 3/2)
};

__device__ __forceinline__ Target2 target2(float4 xi)
{
    return {f2pack(xi.x, xi.x), f2pack(xi.y, xi.y), f2pack(xi.z, xi.z), f2pack(-0.5f, -0.5f),
            f2pack(1.5f, 1.5f)};
}

// The target against two sources (packed x, y, z, q); accumulators packed per source.
__device__ __forceinline__ void p2p_interact2(const Target2 &T, f2 sx, f2 sy, f2 sz, f2 sq, f2 &phi,
                                              f2 &gx, f2 &gy, f2 &gz)
{
    const f2 dx = f2sub(sx, T.x), dy = f2sub(sy, T.y), dz = f2sub(sz, T.z);
    const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    float ra, rb;
    f2unpack(r2, ra, rb);
    f2 y = f2pack(rsqrt_approx(ra), rsqrt_approx(rb));
    const f2 t = f2mul(f2mul(r2, y), y);
    y = f2mul(y, f2fma(T.mhalf, t, T.threehalf));
    float ya, yb;
    f2unpack(y, ya, yb);
    y = f2pack(fmaxf(ya, 0.f), fmaxf(yb, 0.f));
    const f2 qy = f2mul(sq, y);
    phi = f2add(phi, qy);
    const f2 qy3 = f2mul(f2mul(qy, y), y);
    gx = f2fma(qy3, dx, gx);
    gy = f2fma(qy3, dy, gy);
    gz = f2fma(qy3, dz, gz);
}

__device__ __forceinline__ float f2sum(f2 v)
{
    float a, b;
    f2unpack(v, a, b);
    return a + b;
}

__device__ __forceinline__ void p2p_interact(float xi, float yi, float zi, float4 s, float &phi,
                                             float &gx, float &gy, float &gz)
{
    const float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float y = rsqrt_approx(r2);
    const float t = (r2 * y) * y;
    y = y * fmaf(-0.5f, t, 1.5f);
    y = fmaxf(y, 0.f);
    const float qy = s.w * y;
    phi += qy;
    const float qy3 = qy * y * y;
    gx = fmaf(qy3, dx, gx);
    gy = fmaf(qy3, dy, gy);
    gz = fmaf(qy3, dz, gz);
}

}  // namespace

// Stages the next chunk of up to 32 sources of the target's source stream (the
// concatenated particle ranges of its P2P source cells) into sh = x[32], y[32],
// z[32], q[32], padded with zero charges at the origin.  (r, o) = current source
// cell in the list and offset in it; returns false when the stream is exhausted.
__device__ __forceinline__ bool load_chunk(const int *__restrict__ slist, int cnt,
                                           const CellArrays &c, const float4 *__restrict__ pts,
                                           float *sh, int lane, int &r, int &o)
{
    if (r >= cnt) return false;
    const int rk = r + lane;
    int beg = 0, len = 0;
    if (rk < cnt) {
        const int S = slist[rk];
        beg = c.begin[S];
        len = c.end[S] - beg;
    }
    const int ok = lane == 0 ? o : 0;  // already consumed part of the first range
    beg += ok;
    len -= ok;
    int P = len;  // inclusive prefix of remaining lengths
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, P, d);
        if (lane >= d) P += t;
    }
    const int S0 = P - len;  // chunk position where range k starts
    const unsigned starts = __reduce_or_sync(0xffffffffu, (len > 0 && S0 < 32) ? (1u << S0) : 0u);
    const int total = __shfl_sync(0xffffffffu, P, 31);
    const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int k = __popc(starts & le) - 1;
    const int kb = __shfl_sync(0xffffffffu, beg, k), ks = __shfl_sync(0xffffffffu, S0, k);
    const float4 pj = lane < total ? pts[kb + (lane - ks)] : make_float4(0.f, 0.f, 0.f, 0.f);
    sh[lane] = pj.x;
    sh[32 + lane] = pj.y;
    sh[64 + lane] = pj.z;
    sh[96 + lane] = pj.w;
    if (total <= 32) {
        // every range of the window is consumed (a full window of 32 ranges
        // totals at least 32 elements, so fewer than 32 means the list ended)
        r = min(r + 32, cnt);
        o = 0;
    } else {
        // the range holding chunk position 31
        const int k31 = __popc(starts) - 1;
        const int s31 = __shfl_sync(0xffffffffu, S0, k31);
        const int l31 = __shfl_sync(0xffffffffu, len, k31);
        const int o31 = __shfl_sync(0xffffffffu, ok, k31);
        const int used = 32 - s31;  // elements of range k31 consumed in this chunk
        if (used == l31) {
            r += k31 + 1;
            o = 0;
        } else {
            r += k31;
            o = o31 + used;
        }
    }
    return true;
}

// The staged 32 sources against one target: pairs of sources per packed
// instruction, two accumulator sets (sources 4k, 4k+1 and 4k+2, 4k+3).
struct Acc2 {
    f2 phi, gx, gy, gz;
};

__device__ __forceinline__ void p2p_chunk32(const Target2 &T, const float *sh, Acc2 &a, Acc2 &b)
{
#pragma unroll
    for (int jj = 0; jj < 32; jj += 4) {
        const ulonglong2 vx = *reinterpret_cast<const ulonglong2 *>(sh + jj);
        const ulonglong2 vy = *reinterpret_cast<const ulonglong2 *>(sh + 32 + jj);
        const ulonglong2 vz = *reinterpret_cast<const ulonglong2 *>(sh + 64 + jj);
        const ulonglong2 vq = *reinterpret_cast<const ulonglong2 *>(sh + 96 + jj);
        p2p_interact2(T, vx.x, vy.x, vz.x, vq.x, a.phi, a.gx, a.gy, a.gz);
        p2p_interact2(T, vx.y, vy.y, vz.y, vq.y, b.phi, b.gx, b.gy, b.gz);
    }
}

// One warp per target leaf.  Targets go 32 at a time, one per lane; the last
// r <= 16 targets are processed with the 32 staged sources split into
// g = floor(32 / r) contiguous runs of an even length, so that r * g lanes stay
// busy, and the g partial sums are added in shared memory.
__device__ __forceinline__ void p2p_leaf(const CellArrays &c, const ListArrays &L, int T,
                                         const float4 *__restrict__ pts, float4 *__restrict__ near,
                                         float *sh, float4 *redbuf, int lane)
{
    const int b = c.begin[T], e = c.end[T];
    const int *slist = L.p2p_src + L.p2p_off[T];
    const int cnt = L.p2p_cnt[T];
    const f2 zero = 0ull;
    int tb = b;
    // full passes, and a last pass of 17..31 targets (g = 1), one target per lane
    while (tb < e && (e - tb >= 32 || 2 * (e - tb) > 32)) {
        const bool valid = tb + lane < e;
        const Target2 Tg = target2(pts[valid ? tb + lane : tb]);
        Acc2 a0 = {zero, zero, zero, zero}, a1 = a0;
        int r = 0, o = 0;
        while (load_chunk(slist, cnt, c, pts, sh, lane, r, o)) {
            __syncwarp();
            p2p_chunk32(Tg, sh, a0, a1);
            __syncwarp();
        }
        // accumulators hold (phi, gx, gy, gz)
        if (valid)
            near[tb + lane] = make_float4(f2sum(a0.phi) + f2sum(a1.phi), f2sum(a0.gx) + f2sum(a1.gx),
                                          f2sum(a0.gy) + f2sum(a1.gy), f2sum(a0.gz) + f2sum(a1.gz));
        tb += 32;
    }
    const int rem = e - tb;
    if (rem > 0) {
        // 1 <= rem <= 16: g >= 2 runs of cs sources (cs even, g * cs >= 32)
        const int g = 32 / rem;
        const int cs = 2 * ((16 + g - 1) / g);
        const int t = lane % rem, sub = lane / rem;
        const int j0 = sub < g ? sub * cs : 32, j1 = min(32, j0 + cs);
        const Target2 Tg = target2(pts[tb + t]);
        Acc2 a = {zero, zero, zero, zero};
        int r = 0, o = 0;
        while (load_chunk(slist, cnt, c, pts, sh, lane, r, o)) {
            __syncwarp();
#pragma unroll 4
            for (int jj = j0; jj < j1; jj += 2)
                p2p_interact2(Tg, *reinterpret_cast<const f2 *>(sh + jj),
                              *reinterpret_cast<const f2 *>(sh + 32 + jj),
                              *reinterpret_cast<const f2 *>(sh + 64 + jj),
                              *reinterpret_cast<const f2 *>(sh + 96 + jj), a.phi, a.gx, a.gy, a.gz);
            __syncwarp();
        }
        redbuf[lane] = make_float4(f2sum(a.phi), f2sum(a.gx), f2sum(a.gy), f2sum(a.gz));
        __syncwarp();
        if (lane < rem) {
            float4 v0 = redbuf[lane];
            for (int k = 1; k < g; ++k) {
                const float4 v = redbuf[lane + k * rem];
                v0.x += v.x;
                v0.y += v.y;
                v0.z += v.z;
                v0.w += v.w;
            }
            near[tb + lane] = v0;
        }
        __syncwarp();
    }
}

// Persistent: a fixed number of blocks per SM, each warp taking the next leaf
// from a counter, so the kernel leaves room on every SM for the far-field chain
// that runs beside it and has no tail wave.
__global__ void __launch_bounds__(128, kP2PBlocksPerSM)
    k_p2p(CellArrays c, ListArrays L, const int *__restrict__ leaves, int nleaves,
          const float4 *__restrict__ pts, float4 *__restrict__ near, int *__restrict__ counter)
{
    __shared__ __align__(16) float sh[4][128];
    __shared__ float4 red[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(counter, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= nleaves) break;
        p2p_leaf(c, L, leaves[li], pts, near, sh[warp], red[warp], lane);
    }
}

// All-pairs sum: one thread per target, 256-source tiles in shared memory.
__global__ void __launch_bounds__(256)
    k_direct(const float *__restrict__ xyz, const float *__restrict__ q, int64_t n,
             float *__restrict__ phi, float *__restrict__ grad)
{
    __shared__ float4 sh[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const float xi = valid ? xyz[3 * i] : 0.f, yi = valid ? xyz[3 * i + 1] : 0.f,
                zi = valid ? xyz[3 * i + 2] : 0.f;
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    for (int64_t s0 = 0; s0 < n; s0 += 256) {
        const int64_t j = s0 + threadIdx.x;
        sh[threadIdx.x] = j < n ? make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], q[j])
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < 256; ++jj) p2p_interact(xi, yi, zi, sh[jj], ph, gx, gy, gz);
        __syncthreads();
    }
    if (valid) {
        phi[i] = ph;
        grad[3 * i] = gx;
        grad[3 * i + 1] = gy;
        grad[3 * i + 2] = gz;
    }
}

// phi/grad in caller order = far + near of each sorted position.
__global__ void k_combine(const float4 *__restrict__ far, const float4 *__restrict__ near,
                          const uint32_t *__restrict__ idx, int64_t n, float *__restrict__ phi,
                          float *__restrict__ grad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = far[i], b = near[i];
        const uint32_t o = idx[i];
        phi[o] = a.x + b.x;
        grad[3 * (int64_t)o] = a.y + b.y;
        grad[3 * (int64_t)o + 1] = a.z + b.z;
        grad[3 * (int64_t)o + 2] = a.w + b.w;
    }
}

}  // namespace fmm
