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
// concatenated particle ranges of its P2P source leaves) into sh[0..32), padded
// with zero charges.  (r, o) = current source leaf in the list and offset in it;
// returns false when the stream is exhausted.
__device__ __forceinline__ bool load_chunk(const int *__restrict__ slist, int cnt,
                                           const CellArrays &c, const float4 *__restrict__ pts,
                                           float4 *sh, int lane, int &r, int &o)
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
    sh[lane] = lane < total ? pts[kb + (lane - ks)] : make_float4(0.f, 0.f, 0.f, 0.f);
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

// 32 sources from shared memory against one target, two accumulator sets
// (even/odd sources) to shorten the dependency chains.
__device__ __forceinline__ void p2p_chunk32(const float4 &xi, const float4 *buf, float4 &a0, float4 &a1)
{
#pragma unroll
    for (int jj = 0; jj < 32; jj += 2) {
        p2p_interact(xi.x, xi.y, xi.z, buf[jj], a0.x, a0.y, a0.z, a0.w);
        p2p_interact(xi.x, xi.y, xi.z, buf[jj + 1], a1.x, a1.y, a1.z, a1.w);
    }
}

// One warp per target leaf.  Targets go 32 at a time, one per lane; the last
// r <= 16 targets are processed with the sources split into g = floor(32 / r)
// interleaved subsets, so that r * g lanes stay busy, and the g partial sums are
// added in shared memory.
__device__ __forceinline__ void p2p_leaf(const CellArrays &c, const ListArrays &L, int T,
                                         const float4 *__restrict__ pts, float4 *__restrict__ near,
                                         float4 *buf, float4 *redbuf, int lane)
{
    const int b = c.begin[T], e = c.end[T];
    const int *slist = L.p2p_src + L.p2p_off[T];
    const int cnt = L.p2p_cnt[T];
    int tb = b;
    // full passes, and a last pass of 17..31 targets (g = 1), one target per lane
    while (tb < e && (e - tb >= 32 || 2 * (e - tb) > 32)) {
        const bool valid = tb + lane < e;
        const float4 xi = pts[valid ? tb + lane : tb];
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        int r = 0, o = 0;
        while (load_chunk(slist, cnt, c, pts, buf, lane, r, o)) {
            __syncwarp();
            p2p_chunk32(xi, buf, a0, a1);
            __syncwarp();
        }
        // accumulators hold (phi, gx, gy, gz)
        if (valid) near[tb + lane] = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
        tb += 32;
    }
    const int rem = e - tb;
    if (rem > 0) {
        // 1 <= rem <= 16: g >= 2 interleaved source subsets
        const int g = 32 / rem;
        const int t = lane % rem, sub = lane / rem;
        const bool active = sub < g;
        const float4 xi = pts[tb + t];
        float phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        int r = 0, o = 0;
        while (load_chunk(slist, cnt, c, pts, buf, lane, r, o)) {
            __syncwarp();
            if (active) {
#pragma unroll 4
                for (int jj = sub; jj < 32; jj += g) p2p_interact(xi.x, xi.y, xi.z, buf[jj], phi, gx, gy, gz);
            }
            __syncwarp();
        }
        redbuf[lane] = make_float4(phi, gx, gy, gz);
        __syncwarp();
        if (lane < rem) {
            float4 a = redbuf[lane];
            for (int k = 1; k < g; ++k) {
                const float4 v = redbuf[lane + k * rem];
                a.x += v.x;
                a.y += v.y;
                a.z += v.z;
                a.w += v.w;
            }
            near[tb + lane] = a;
        }
        __syncwarp();
    }
}

// Persistent: a fixed number of blocks per SM, each warp taking the next leaf
// from a counter, so the kernel leaves room on every SM for the far-field chain
// that runs beside it and has no tail wave.
__global__ void __launch_bounds__(128)
    k_p2p(CellArrays c, ListArrays L, const int *__restrict__ leaves, int nleaves,
          const float4 *__restrict__ pts, float4 *__restrict__ near, int *__restrict__ counter)
{
    __shared__ float4 sh[4][32];
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
