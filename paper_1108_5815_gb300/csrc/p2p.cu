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

// One warp per target leaf, 4 warps per block.
__global__ void __launch_bounds__(128)
    k_p2p(CellArrays c, ListArrays L, const int *__restrict__ leaves, int nleaves,
          const float4 *__restrict__ pts, float4 *__restrict__ near)
{
    __shared__ float4 sh[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * 4 + warp;
    if (li >= nleaves) return;
    const int T = leaves[li];
    const int b = c.begin[T], e = c.end[T];
    const int off = L.p2p_off[T], cnt = L.p2p_cnt[T];
    for (int tb = b; tb < e; tb += 32) {
        const int i = tb + lane;
        const bool valid = i < e;
        const float4 xi = valid ? pts[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int k = 0; k < cnt; ++k) {
            const int S = L.p2p_src[off + k];
            const int sb = c.begin[S], se = c.end[S];
            for (int s0 = sb; s0 < se; s0 += 32) {
                const int j = s0 + lane;
                sh[warp][lane] = j < se ? pts[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj)
                    p2p_interact(xi.x, xi.y, xi.z, sh[warp][jj], phi, gx, gy, gz);
                __syncwarp();
            }
        }
        if (valid) near[i] = make_float4(phi, gx, gy, gz);
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
