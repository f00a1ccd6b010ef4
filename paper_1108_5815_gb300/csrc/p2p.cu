// p2p.cu -- particle-particle near field, the all-pairs direct sum, and the
// final combination of near and far fields in the caller's order.
//
// P2P (the paper's "local evaluation", which dominates its GPU run time,
// Fig. "breakdown") sums q_j / r and q_j (x_j - x_i) / r^3 over the sources of
// the target leaf's P2P list.  Target-parallel (one lane per target particle,
// the layout of Nyland et al. that the paper recounts): no reduction across
// threads, source tiles staged through shared memory and broadcast.
//
// Per interaction: 3 FADD for the offset, 3 for r^2, one MUFU rsqrt y0 and one
// Newton step y = y0 (3 - r^2 y0^2) / 2, then phi += q y and grad += q y^3 d.
// The step is taken without its factor -1/2: z = y0 (r^2 y0^2 - 3) = -2 y is
// three operations (t = y0^2, one FMA, one product), the charge is staged as
// -q/2 so that u = (-q/2) z = q y and phi += u, and the gradient's weight is
// w = u t = q y y0^2: the Newton-refined 1/r times the 1/r^2 that the step has
// already formed from y0 (relative error within twice the rsqrt's), and
// grad += w d.  15 FP32-pipe lane operations per interaction (17 with a
// separate -1/2 and y^3 = y y y).  Pairs at r = 0 (the particle itself,
// coincident points) contribute nothing: rsqrt(0) = inf makes the Newton step
// NaN and min(NaN, 0) = 0 removes it without a branch (valid z are negative),
// and t = inf is clamped to the largest float so that w = 0 * t stays 0.
// Only a chunk holding sources of
// the target's own leaf can hold the particle itself, so only those chunks take
// the guard; a pass that still ends with a non-finite sum (a pair at r = 0 in
// two leaves, r^2 flushed to zero, a target at the origin meeting the zero
// padding, overflow) is run again with the guard on every chunk, which gives
// exactly the result of guarding every pair.
// Each lane takes its target against two sources at a time with the packed
// FP32x2 instructions (add/sub/mul/fma.rn.f32x2): one instruction does the same
// operation for both sources, which halves the issue slots of the arithmetic;
// only the rsqrt and the NaN guard stay scalar.  Sources are staged in shared
// memory as four arrays (x, y, z, q), so a pair of consecutive sources is one
// 64-bit load per component.
#include <cfloat>

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
    f2 x, y, z;  // the target's coordinates in both halves
    f2 mthree;   // (-3, -3)
};

__device__ __forceinline__ Target2 target2(float4 xi)
{
    return {f2pack(xi.x, xi.x), f2pack(xi.y, xi.y), f2pack(xi.z, xi.z), f2pack(-3.f, -3.f)};
}

// The target against two sources (packed x, y, z and staged charge -q/2);
// accumulators packed per source: phi and grad.
template <bool GUARD>
__device__ __forceinline__ void p2p_interact2(const Target2 &T, f2 sx, f2 sy, f2 sz, f2 sqn, f2 &phi,
                                              f2 &gx, f2 &gy, f2 &gz)
{
    const f2 dx = f2sub(sx, T.x), dy = f2sub(sy, T.y), dz = f2sub(sz, T.z);
    const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    float ra, rb;
    f2unpack(r2, ra, rb);
    const f2 y0 = f2pack(rsqrt_approx(ra), rsqrt_approx(rb));
    f2 t = f2mul(y0, y0);                  // 1 / r^2 (unrefined)
    f2 z = f2mul(y0, f2fma(r2, t, T.mthree));  // -2 y
    if (GUARD) {
        float za, zb, ta, tb;
        f2unpack(z, za, zb);
        f2unpack(t, ta, tb);
        z = f2pack(fminf(za, 0.f), fminf(zb, 0.f));
        t = f2pack(fminf(ta, FLT_MAX), fminf(tb, FLT_MAX));
    }
    const f2 u = f2mul(sqn, z);  // q y
    phi = f2add(phi, u);
    const f2 w = f2mul(u, t);  // q y^3
    gx = f2fma(w, dx, gx);
    gy = f2fma(w, dy, gy);
    gz = f2fma(w, dz, gz);
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

// The source stream of a target leaf is the particle ranges of its P2P list
// concatenated in list order and cut into chunks of 32.  A window holds up to 32
// consecutive list entries, one per lane: the first particle of the entry's
// range and where the range starts and ends in the window's part of the stream.
struct Window {
    int beg, start, end;  // this lane's entry
    int total;            // particles in the window
};

__device__ __forceinline__ Window load_window(const int *__restrict__ slist, int cnt, int r0,
                                              const CellArrays &c, int lane)
{
    const int rk = r0 + lane;
    int beg = 0, len = 0;
    if (rk < cnt) {
        const int S = slist[rk];
        beg = c.begin[S];
        len = c.end[S] - beg;
    }
    int P = len;  // inclusive prefix of the lengths
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, P, d);
        if (lane >= d) P += t;
    }
    return {beg, P - len, P, __shfl_sync(0xffffffffu, P, 31)};
}

// The particle at window position pos (0 <= pos < total): the entry k whose
// range holds pos is the first lane with end > pos, found by a binary search
// over the lanes.  Every lane takes part; for pos >= total the result is not
// an index and must not be used.
__device__ __forceinline__ int window_particle(const Window &w, int pos)
{
    int k = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(0xffffffffu, w.end, k + step - 1) <= pos) k += step;
    return __shfl_sync(0xffffffffu, w.beg, k) + (pos - __shfl_sync(0xffffffffu, w.start, k));
}

// Sources at window positions s .. s+31, one per lane, zero charges at the
// origin past the end; own = one of them lies in [own_b, own_e).
__device__ __forceinline__ float4 fetch_chunk(const Window &w, int s, const float4 *__restrict__ pts, int lane,
                                              int own_b, int own_e, bool &own)
{
    const int pos = s + lane;
    const int j = window_particle(w, pos);
    const bool in = pos < w.total;
    own = __any_sync(0xffffffffu, in && j >= own_b && j < own_e);
    return in ? pts[j] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The staged 32 sources (x, y, z, -q/2) against one target: pairs of sources
// per packed instruction, two accumulator sets (sources 4k, 4k+1 and 4k+2, 4k+3).
struct Acc2 {
    f2 phi, gx, gy, gz;
};

template <bool GUARD>
__device__ __forceinline__ void p2p_chunk32(const Target2 &T, const float *sh, Acc2 &a, Acc2 &b)
{
#pragma unroll
    for (int jj = 0; jj < 32; jj += 4) {
        const ulonglong2 vx = *reinterpret_cast<const ulonglong2 *>(sh + jj);
        const ulonglong2 vy = *reinterpret_cast<const ulonglong2 *>(sh + 32 + jj);
        const ulonglong2 vz = *reinterpret_cast<const ulonglong2 *>(sh + 64 + jj);
        const ulonglong2 vq = *reinterpret_cast<const ulonglong2 *>(sh + 96 + jj);
        p2p_interact2<GUARD>(T, vx.x, vy.x, vz.x, vq.x, a.phi, a.gx, a.gy, a.gz);
        p2p_interact2<GUARD>(T, vx.y, vy.y, vz.y, vq.y, b.phi, b.gx, b.gy, b.gz);
    }
}

// One run of sources [j0, j1) of the staged chunk (j1 - j0 even).
template <bool GUARD>
__device__ __forceinline__ void p2p_run(const Target2 &T, const float *sh, int j0, int j1, Acc2 &a)
{
#pragma unroll 4
    for (int jj = j0; jj < j1; jj += 2)
        p2p_interact2<GUARD>(T, *reinterpret_cast<const f2 *>(sh + jj), *reinterpret_cast<const f2 *>(sh + 32 + jj),
                             *reinterpret_cast<const f2 *>(sh + 64 + jj), *reinterpret_cast<const f2 *>(sh + 96 + jj),
                             a.phi, a.gx, a.gy, a.gz);
}

// phi and grad of one accumulator set
__device__ __forceinline__ float4 acc_sum(const Acc2 &a)
{
    return make_float4(f2sum(a.phi), f2sum(a.gx), f2sum(a.gy), f2sum(a.gz));
}

__device__ __forceinline__ bool nonfinite(float4 v)
{
    return !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
}

// One warp per target leaf; one walk of the source stream serves up to 64
// targets.  Group A, the first min(n, 32) targets when there are more than 16,
// takes one target per lane against all 32 sources of each chunk.  Group B,
// the next up to 32: with more than 16 targets one per lane as well; with
// r <= 16 the 32 sources of a chunk are split into g = floor(32 / r) runs of
// an even length so that r * g lanes stay busy, and the g partial sums are
// added in shared memory.
__device__ __forceinline__ void p2p_leaf(const CellArrays &c, const ListArrays &L, int T,
                                         const float4 *__restrict__ pts, float4 *__restrict__ near,
                                         float *sh, float4 *redbuf, int lane)
{
    const int b = c.begin[T], e = c.end[T];
    const int *slist = L.p2p_src + L.p2p_off[T];
    const int cnt = L.p2p_cnt[T];
    const f2 zero = 0ull;
    bool guard_all = false;  // set once a pass has produced a non-finite sum
    for (int tb = b; tb < e;) {
        const int n = e - tb;
        const int nA = n > 16 ? min(n, 32) : 0;
        const int nB = min(n - nA, 32);
        const bool bfull = nB > 16;
        int g = 1, t = lane, j0 = 0, j1 = 0;
        if (nB > 0 && !bfull) {
            g = 32 / nB;
            const int cs = 2 * ((16 + g - 1) / g);
            t = lane % nB;
            const int sub = lane / nB;
            j0 = sub < g ? sub * cs : 32;
            j1 = min(32, j0 + cs);
        }
        const Target2 TA = target2(pts[lane < nA ? tb + lane : tb]);
        const Target2 TB = target2(pts[nB > 0 && t < nB ? tb + nA + t : tb]);
        Acc2 a0 = {zero, zero, zero, zero}, a1 = a0, ab = a0;
        for (int r0 = 0; r0 < cnt; r0 += 32) {
            const Window w = load_window(slist, cnt, r0, c, lane);
            bool own_next;
            float4 nx = fetch_chunk(w, 0, pts, lane, b, e, own_next);
            for (int s = 0; s < w.total; s += 32) {
                const bool guard = own_next || guard_all;
                sh[lane] = nx.x;
                sh[32 + lane] = nx.y;
                sh[64 + lane] = nx.z;
                sh[96 + lane] = -0.5f * nx.w;
                __syncwarp();
                if (s + 32 < w.total) nx = fetch_chunk(w, s + 32, pts, lane, b, e, own_next);
                if (guard) {
                    if (nA > 0) p2p_chunk32<true>(TA, sh, a0, a1);
                    if (bfull) p2p_run<true>(TB, sh, 0, 32, ab);
                    else if (nB > 0) p2p_run<true>(TB, sh, j0, j1, ab);
                } else {
                    if (nA > 0) p2p_chunk32<false>(TA, sh, a0, a1);
                    if (bfull) p2p_run<false>(TB, sh, 0, 32, ab);
                    else if (nB > 0) p2p_run<false>(TB, sh, j0, j1, ab);
                }
                __syncwarp();
            }
        }
        float4 va = acc_sum(a0);
        const float4 va1 = acc_sum(a1);
        va.x += va1.x;
        va.y += va1.y;
        va.z += va1.z;
        va.w += va1.w;
        const float4 vb = acc_sum(ab);
        const bool bad = (lane < nA && nonfinite(va)) || (nB > 0 && (bfull ? lane < nB : true) && nonfinite(vb));
        if (!guard_all && __any_sync(0xffffffffu, bad)) {
            // a pair at r = 0 outside the target's own leaf, r^2 flushed to zero,
            // or a non-finite input: the same pass again with every chunk guarded
            guard_all = true;
            continue;
        }
        if (lane < nA) near[tb + lane] = va;
        if (bfull) {
            if (lane < nB) near[tb + nA + lane] = vb;
        } else if (nB > 0) {
            redbuf[lane] = vb;
            __syncwarp();
            if (lane < nB) {
                float4 v0 = redbuf[lane];
                for (int k = 1; k < g; ++k) {
                    const float4 v = redbuf[lane + k * nB];
                    v0.x += v.x;
                    v0.y += v.y;
                    v0.z += v.z;
                    v0.w += v.w;
                }
                near[tb + nA + lane] = v0;
            }
            __syncwarp();
        }
        tb += nA + nB;
    }
}

// One 32-thread block per target leaf (leaves[blockIdx.x]), up to
// kP2PWarpsPerSM resident per SM with 128 registers a thread.  Blocks retire as
// their leaves finish, so kernels of the far-field stream, which has the higher
// priority, take SMs while P2P runs, and the M2L kernel starts on the SMs that
// P2P has drained.
__global__ void __launch_bounds__(32, kP2PWarpsPerSM)
    k_p2p(CellArrays c, ListArrays L, const int *__restrict__ leaves, int nleaves,
          const float4 *__restrict__ pts, float4 *__restrict__ near, const int *__restrict__ sz)
{
    if (sz) nleaves = sz[kSzLeaves];
    __shared__ __align__(16) float sh[128];
    __shared__ float4 red[32];
    const int li = blockIdx.x;
    if (li >= nleaves) return;
    p2p_leaf(c, L, leaves[li], pts, near, sh, red, threadIdx.x);
}

// Ceilings of the FP32 pipe on this device, for the P2P roofline.
//
// k_ffma_stream: eight independent FP32x2 FMA chains per thread, nothing else
// in the loop -- the rate the FMA pipe sustains.  k_p2p_body: the P2P kernel's
// own interaction code (p2p_chunk32, unguarded) on 32 sources staged once in
// shared memory, `reps` passes, no list walk and no global loads -- the rate of
// the interaction body alone.  Both write one value per thread so that the work
// is kept.
__global__ void __launch_bounds__(256) k_ffma_stream(float *__restrict__ out, int iters, float s)
{
    f2 a[8];
    const f2 m = f2pack(s, s), c = f2pack(0.5f * s, 0.25f * s);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = f2pack(threadIdx.x * 1e-3f + k, k * 0.1f);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = f2fma(a[k], m, c);
    }
    float x = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) x += f2sum(a[k]);
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

__global__ void __launch_bounds__(128, kP2PBlocksPerSM) k_p2p_body(float *__restrict__ out, int reps)
{
    __shared__ __align__(16) float sh[4][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *s = sh[warp];
    s[lane] = 0.37f * lane;
    s[32 + lane] = 0.11f * lane + 0.5f;
    s[64 + lane] = 0.05f * lane - 0.3f;
    s[96 + lane] = -0.5f / (1 + lane);
    __syncwarp();
    const Target2 T = target2(make_float4(0.013f * threadIdx.x + 40.f, 0.2f, -0.1f, 0.f));
    const f2 zero = 0ull;
    Acc2 a0 = {zero, zero, zero, zero}, a1 = a0;
#pragma unroll 1
    for (int r = 0; r < reps; ++r) {
        __syncwarp();
        p2p_chunk32<false>(T, s, a0, a1);
        __syncwarp();
        if (lane == 0 && r < 0) s[0] = 1.f;  // never: the staged sources may change as far as the compiler knows
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] =
        f2sum(a0.phi) + f2sum(a1.phi) + f2sum(a0.gx) + f2sum(a1.gx) + f2sum(a0.gy) + f2sum(a1.gy) + f2sum(a0.gz) +
        f2sum(a1.gz);
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
                          float *__restrict__ grad, const IoPtrs *__restrict__ io)
{
    if (io) {
        phi = io->phi;
        grad = io->grad;
    }
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
