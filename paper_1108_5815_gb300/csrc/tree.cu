// tree.cu -- bounding box, Morton keys, particle permutation and the adaptive
// octree, built level by level on the GPU.
//
// The paper builds its adaptive tree (at most N_crit particles per cell,
// Results section) on the host CPU; here every step runs on the device.
// Quantisation follows the FP64 reading documented in the header: the box is
// the cube [lo, lo + side) with side the largest extent, a coordinate maps to
// k = min(2^21 - 1, floor((x - lo) * (2^21 / side))) with each operation a single
// IEEE round-to-nearest FP64 operation (__dsub_rn/__dmul_rn/__ddiv_rn, no
// contraction), so keys match an FP64 CPU computation bit for bit.
#include <climits>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ uint32_t float_to_ordered(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float ordered_to_float(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

}  // namespace

// bbox_u[0..2] = ordered min, [3..5] = ordered max; flags[kFlagNonfinite] set on NaN/Inf.
__global__ void k_bbox(const float *__restrict__ xyz, int64_t n, uint32_t *__restrict__ bbox_u,
                       int *__restrict__ flags, const IoPtrs *__restrict__ io)
{
    if (io) xyz = io->xyz;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float v = xyz[3 * i + a];
            bad |= !isfinite(v);
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    // one set of atomics per block: the warps' results meet in shared memory first
    __shared__ float smn[3][32], smx[3][32];
    __shared__ int sbad;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            smn[a][warp] = mn[a];
            smx[a][warp] = mx[a];
        }
        if (bad) sbad = 1;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        float bmn = smn[a][0], bmx = smx[a][0];
        for (int w = 1; w < nw; ++w) {
            bmn = fminf(bmn, smn[a][w]);
            bmx = fmaxf(bmx, smx[a][w]);
        }
        atomicMin(&bbox_u[a], float_to_ordered(bmn));
        atomicMax(&bbox_u[3 + a], float_to_ordered(bmx));
    }
    if (threadIdx.x == 0 && sbad) atomicOr(&flags[kFlagNonfinite], 1);
}

// System of particle i: the s with off[s] <= i < off[s+1].
__device__ __forceinline__ int system_of(const int *__restrict__ off, int nsys, int64_t i)
{
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Box of one system from its ordered min/max: lo per axis and the cube side.
__device__ __forceinline__ void decode_box(const uint32_t *__restrict__ bu, double lo[3], double &side)
{
    side = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)ordered_to_float(bu[a]);
        const double hi = (double)ordered_to_float(bu[3 + a]);
        const double ext = __dsub_rn(hi, lo[a]);
        side = ext > side ? ext : side;
    }
    if (!(side > 0.0)) side = 1.0;
}

// Per-system box for several systems stored back to back (off[] on the device):
// each thread reduces 8 consecutive particles, flushing when the system changes;
// a warp whose lanes end in one system combines before its atomics.
__global__ void k_bbox_sys(const float *__restrict__ xyz, int64_t n, const int *__restrict__ off,
                           int nsys, uint32_t *__restrict__ bbox_u, int *__restrict__ flags,
                           const IoPtrs *__restrict__ io)
{
    if (io) xyz = io->xyz;
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    int cur = i0 < n ? system_of(off, nsys, i0) : -1;
    for (int64_t i = i0; i < n && i < i0 + 8; ++i) {
        if (i >= off[cur + 1]) {
            for (int a = 0; a < 3; ++a) {
                atomicMin(&bbox_u[6 * cur + a], float_to_ordered(mn[a]));
                atomicMax(&bbox_u[6 * cur + 3 + a], float_to_ordered(mx[a]));
                mn[a] = INFINITY;
                mx[a] = -INFINITY;
            }
            while (i >= off[cur + 1]) ++cur;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * i + a];
            bad |= !isfinite(v);
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
    const int s0 = __shfl_sync(0xffffffffu, cur, 0);
    const bool uniform = __all_sync(0xffffffffu, cur == s0 || cur < 0);
    if (uniform) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
            }
    }
    if (cur >= 0 && (!uniform || (threadIdx.x & 31) == 0)) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bbox_u[6 * cur + a], float_to_ordered(mn[a]));
            atomicMax(&bbox_u[6 * cur + 3 + a], float_to_ordered(mx[a]));
        }
    }
    if (bad) atomicOr(&flags[kFlagNonfinite], 1);
}

// Key quantisation k = floor(fl64(fl64(x - lo) * s)), clamped to [0, 2^21 - 1]
// (FP64, one rounding per operation), taken in FP32 arithmetic when that
// decides it: the difference x - lo of two floats is exact as dh + dl (TwoSum)
// and is exact in FP64 when their exponents differ by at most 28; with
// s = s_hi + s_lo, p + e = (dh + dl)(s_hi + s_lo) (TwoProd for dh s_hi) is
// within 2^-44 relative (2^-23 absolute below 2^21) of the FP64 product, so
// floor() is decided whenever p + e lies more than 2^-20 from an integer.
// Otherwise (false) the caller takes the FP64 operations themselves.
__device__ __forceinline__ bool quant_fast(float x, float lo, float s_hi, float s_lo, uint32_t &k)
{
    const float b = -lo;
    const float dh = __fadd_rn(x, b);
    const float bv = __fsub_rn(dh, x), av = __fsub_rn(dh, bv);
    const float br = __fsub_rn(b, bv), ar = __fsub_rn(x, av);
    const float dl = __fadd_rn(ar, br);
    const int ex = (__float_as_int(x) >> 23) & 0xff, el = (__float_as_int(lo) >> 23) & 0xff;
    if (!(x == 0.f || lo == 0.f || abs(ex - el) <= 28)) return false;
    const float p = __fmul_rn(dh, s_hi);
    const float e1 = __fmaf_rn(dh, s_hi, -p);
    const float e2 = __fmaf_rn(dh, s_lo, __fmul_rn(dl, s_hi));
    const float e = __fadd_rn(e1, e2);
    const float k0 = floorf(p);
    const float r = __fadd_rn(__fsub_rn(p, k0), e);
    const float m = 9.5367431640625e-07f;  // 2^-20
    float kf;
    if (r > m && r < 1.f - m)
        kf = k0;
    else if (r > -1.f + m && r < -m)
        kf = k0 - 1.f;
    else if (r > 1.f + m && r < 2.f - m)
        kf = k0 + 1.f;
    else
        return false;
    k = (uint32_t)fminf(fmaxf(kf, 0.f), 2097151.f);
    return true;
}

// The same with the FP64 operations.
__device__ __forceinline__ uint32_t quant_fp64(float x, double lo, double s)
{
    const double t = __dsub_rn((double)x, lo);
    double f = floor(__dmul_rn(t, s));
    // NaN/Inf inputs are reported through the flag; keep the key in range.
    if (!(f >= 0.0)) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    return (uint32_t)f;
}

// Decodes each system's box into box[4s..4s+3] = lo, side (FP64), then writes
// keys (quantised in the particle's own system box) and the identity permutation.
__global__ void k_morton(const float *__restrict__ xyz, int64_t n, const int *__restrict__ off,
                         int nsys, const uint32_t *__restrict__ bbox_u, double *__restrict__ box,
                         uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, const IoPtrs *__restrict__ io)
{
    if (io) xyz = io->xyz;
    if (blockIdx.x == 0) {
        for (int sy = threadIdx.x; sy < nsys; sy += blockDim.x) {
            double lo[3], side;
            decode_box(bbox_u + 6 * sy, lo, side);
            box[4 * sy] = lo[0];
            box[4 * sy + 1] = lo[1];
            box[4 * sy + 2] = lo[2];
            box[4 * sy + 3] = side;
        }
    }
    // the first system's box and scale 2^21 / side, once per block (FP64 is a slow
    // pipe here): lo per axis (floats), the scale in FP64 and as FP32 hi + lo
    __shared__ double s_scale;
    __shared__ float s_lof[3], s_shi, s_slo;
    if (threadIdx.x == 0) {
        double lo[3], side;
        decode_box(bbox_u, lo, side);
        const double sc = __ddiv_rn(2097152.0, side);
        s_scale = sc;
        s_shi = (float)sc;
        s_slo = (float)(sc - (double)s_shi);
        for (int a = 0; a < 3; ++a) s_lof[a] = (float)lo[a];
    }
    __syncthreads();
    int sys = 0;
    double s = s_scale;
    float lof[3] = {s_lof[0], s_lof[1], s_lof[2]}, s_hi = s_shi, s_lo = s_slo;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (nsys > 1) {
            const int si = system_of(off, nsys, i);
            if (si != sys) {
                sys = si;
                double lo[3], side;
                decode_box(bbox_u + 6 * sys, lo, side);
                s = __ddiv_rn(2097152.0, side);
                s_hi = (float)s;
                s_lo = (float)(s - (double)s_hi);
                for (int a = 0; a < 3; ++a) lof[a] = (float)lo[a];
            }
        }
        uint32_t k[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float x = xyz[3 * i + a];
            if (!quant_fast(x, lof[a], s_hi, s_lo, k[a])) k[a] = quant_fp64(x, (double)lof[a], s);
        }
        keys[i] = spread3_dev(k[0]) | (spread3_dev(k[1]) << 1) | (spread3_dev(k[2]) << 2);
        idx[i] = (uint32_t)i;
    }
}

// Sorted particles as float4 (x, y, z, q).
__global__ void k_permute(const float *__restrict__ xyz, const float *__restrict__ q,
                          const uint32_t *__restrict__ idx, int64_t n, float4 *__restrict__ out,
                          const IoPtrs *__restrict__ io)
{
    if (io) {
        xyz = io->xyz;
        q = io->q;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = idx[i];
        out[i] = make_float4(xyz[3 * o], xyz[3 * o + 1], xyz[3 * o + 2], q[o]);
    }
}

// Second sort key of a batch: the system of each (key-sorted) particle.
__global__ void k_sys_of_sorted(const uint32_t *__restrict__ idx, int64_t n, const int *__restrict__ off,
                                int nsys, uint64_t *__restrict__ sys_key)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        sys_key[i] = (uint64_t)system_of(off, nsys, idx[i]);
}

__global__ void k_gather_keys(const uint64_t *__restrict__ orig, const uint32_t *__restrict__ idx,
                              int64_t n, uint64_t *__restrict__ keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = orig[idx[i]];
}

// One root cell per system; roots fill the first ceil(nsys / 128) M2L tiles.
// Per-system bounding boxes before the reduction: minima at all ones, maxima at zero
// (order-preserving unsigned images of the coordinates).
__global__ void k_init_bbox(uint32_t *bbox_u, int nsys)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 6 * nsys; i += gridDim.x * blockDim.x)
        bbox_u[i] = (i % 6) < 3 ? 0xffffffffu : 0u;
}

__global__ void k_init_roots(CellArrays c, const int *__restrict__ off, int nsys)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
        c.level[s] = 0;
        c.prefix[s] = 0;
        c.begin[s] = off[s];
        c.end[s] = off[s + 1];
        c.parent[s] = -1;
        c.child0[s] = -1;
        c.nchild[s] = 0;
        c.tile[s] = s / kTile;
        c.lane[s] = s % kTile;
        c.sys[s] = s;
    }
}

// Boundary levels: for i in [1, n), the first level at which the keys of
// sorted positions i-1 and i differ (22 when they are equal).  Inside a cell
// of level l every adjacent pair shares the level-l prefix, so the children's
// boundaries are exactly the positions of level l+1 in the cell's range.
__global__ void k_first_diff(const uint64_t *__restrict__ keys, int64_t n,
                             uint64_t *__restrict__ lvl, uint32_t *__restrict__ pos)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = keys[i] ^ keys[i - 1];
        lvl[i - 1] = x ? (uint64_t)(kKeyBits - (63 - __clzll((long long)x)) / 3) : 22ull;
        pos[i - 1] = (uint32_t)i;
    }
}

// start[L] = first index of level L in the (stably) level-sorted boundary list.
// Warp L searches for it 32 probes at a time: each round narrows [lo, hi) to one
// of 32 equal steps, so a million entries take four dependent loads, not twenty.
__global__ void k_level_starts(const uint64_t *__restrict__ lvl, int64_t n, int *__restrict__ start)
{
    const int L = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (L >= kLevelStartWarps) return;
    int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t pos = lo + lane * step;
        const bool below = pos < hi && lvl[pos] < (uint64_t)L;
        const int c = __popc(__ballot_sync(0xffffffffu, below));  // probes below L: a prefix
        if (c == 0) {
            hi = lo;
        } else {
            const int64_t last = lo + (int64_t)(c - 1) * step;  // the last probe below L
            hi = min(hi, last + step);
            lo = last + 1;
        }
    }
    const int64_t pos = lo + lane;
    const bool below = pos < hi && lvl[pos] < (uint64_t)L;
    const int c = __popc(__ballot_sync(0xffffffffu, below));
    if (lane == 0) start[L] = (int)(lo + c);
}

// The first positions of B[0, nb) (ascending) holding a value >= v1 and >= v2,
// in one loop: both probes of a step are loaded before either is compared, so
// the two searches cost the latency of one.
__device__ __forceinline__ void lower_pos2(const uint32_t *__restrict__ B, int nb, uint32_t v1, uint32_t v2, int &r1,
                                           int &r2)
{
    int lo1 = 0, hi1 = nb, lo2 = 0, hi2 = nb;
    while (lo1 < hi1 || lo2 < hi2) {
        const int m1 = (lo1 + hi1) >> 1, m2 = (lo2 + hi2) >> 1;
        const uint32_t x1 = lo1 < hi1 ? B[m1] : 0u, x2 = lo2 < hi2 ? B[m2] : 0u;
        if (lo1 < hi1) {
            if (x1 < v1)
                lo1 = m1 + 1;
            else
                hi1 = m1;
        }
        if (lo2 < hi2) {
            if (x2 < v2)
                lo2 = m2 + 1;
            else
                hi2 = m2;
        }
    }
    r1 = lo1;
    r2 = lo2;
}

// For the cells [a, b) at level l: packed[c-a] = nchild | (split ? 1 << 32 : 0).
// A split cell's child0 holds, until its children are written, the index of
// its first child boundary in the level's boundary list (the emit step reads it
// back instead of searching again).
__global__ void k_split_count(CellArrays c, const uint32_t *__restrict__ bpos,
                              const int *__restrict__ lstart, int a, int b, int level, int ncrit,
                              int max_depth, int64_t *__restrict__ packed, const int *__restrict__ sz, int len)
{
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
    } else {
        len = b - a;
    }
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const int i = a + k;
    if (i >= b) {
        packed[k] = 0;  // past the level: nothing to split
        return;
    }
    const int cb = c.begin[i], ce = c.end[i];
    int64_t v = 0;
    if (ce - cb > ncrit && level < max_depth) {
        const uint32_t *B = bpos + lstart[level + 1];
        const int nb = lstart[level + 2] - lstart[level + 1];
        int lo, hi;
        lower_pos2(B, nb, (uint32_t)cb + 1, (uint32_t)ce, lo, hi);
        v = (int64_t)(hi - lo + 1) | ((int64_t)1 << 32);
        c.child0[i] = lo;
    }
    packed[i - a] = v;
}

// Writes the nch (<= 8) children of cell i (level l, particles [cb, ce)) at
// cells first .. first + nch - 1.  B[lo .. lo + nch - 2] are the boundaries
// between them; all boundaries, then all first keys, are loaded at once (two
// memory latencies per cell, not two per child).
__device__ __forceinline__ void emit_children(CellArrays &c, const uint64_t *__restrict__ keys,
                                              const uint32_t *__restrict__ B, int lo, int i, int level, int cb,
                                              int ce, int nch, int first, int tile, int lane)
{
    const int shift = 3 * (kKeyBits - level - 1);
    const uint64_t pre = c.prefix[i];
    const int sys = c.sys[i];
    int end[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) end[q] = q + 1 < nch ? (int)B[lo + q] : ce;
    int oct[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) oct[q] = q < nch ? (int)((keys[q == 0 ? cb : end[q - 1]] >> shift) & 7ull) : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= nch) break;
        const int ch = first + q, o = oct[q];
        c.level[ch] = level + 1;
        c.prefix[ch] = (pre << 3) | (uint64_t)o;
        c.begin[ch] = q == 0 ? cb : end[q - 1];
        c.end[ch] = end[q];
        c.parent[ch] = i;
        c.child0[ch] = -1;
        c.nchild[ch] = 0;
        c.tile[ch] = tile + o;
        c.lane[ch] = lane;
        c.sys[ch] = sys;
    }
    c.child0[i] = first;
    c.nchild[i] = nch;
}

// Writes the children of the cells [a, b) (level l) starting at cell index b,
// using the exclusive scan `ex` of the packed counts; assigns each child its
// M2L tile (parent window of kTile split parents x octant) and lane.
__global__ void k_split_emit(CellArrays c, const uint64_t *__restrict__ keys,
                             const uint32_t *__restrict__ bpos, const int *__restrict__ lstart,
                             int a, int b, int level, const int64_t *__restrict__ packed,
                             const int64_t *__restrict__ ex, int tile_base, const int *__restrict__ sz)
{
    int cend = INT_MAX;  // children must end before the next level's end
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
        tile_base = sz[kSzTileBase + level];
        cend = sz[kSzLevel + level + 2];
    }
    const int i = a + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b) return;
    const int64_t v = packed[i - a];
    const int64_t e = ex[i - a];
    const int first = b + (int)(e & 0xffffffffll);
    if (v == 0 || first + (int)(v & 0xffffffffll) > cend) {
        // a leaf (or, after a capacity overflow of a replayed plan, kept as one)
        c.child0[i] = -1;
        c.nchild[i] = 0;
        return;
    }
    const int rank = (int)(e >> 32);
    const int window = rank / kTile, lane = rank % kTile;
    const int cb = c.begin[i], ce = c.end[i];
    const uint32_t *B = bpos + lstart[level + 1];
    const int lo = c.child0[i];  // left there by k_split_count
    emit_children(c, keys, B, lo, i, level, cb, ce, (int)(v & 0xffffffffll), first, tile_base + window * 8, lane);
}

// Next level of a replayed plan: the children of level `level` start at the
// level's end; the tiles of their windows follow the tiles so far.  Past a
// capacity the level gets no children (its cells stay leaves) and kSzAbort is
// set.  One thread.
__global__ void k_level_advance(const int64_t *__restrict__ total, int level, int last_level, int cell_cap,
                                int next_level_cap, int tile_cap, int *__restrict__ sz)
{
    const int b = sz[kSzLevel + level + 1];
    const int64_t t = *total;
    const int nch = (int)(t & 0xffffffffll), nsplit = (int)(t >> 32);
    const int tiles = sz[kSzTiles] + 8 * (int)((nsplit + kTile - 1) / kTile);
    sz[kSzTileBase + level] = sz[kSzTiles];
    if (nch > 0 && (level >= last_level || nch > next_level_cap || b + nch > cell_cap || tiles > tile_cap)) {
        sz[kSzAbort] = 1;
        sz[kSzLevel + level + 2] = b;
        return;
    }
    sz[kSzLevel + level + 2] = b + nch;
    sz[kSzTiles] = tiles;
    sz[kSzCells] = b + nch;
}

// The first levels of a tree built with device-side level ranges (capacities
// from an earlier solve), in one block: level l = 0 .. sl.n - 1 takes the steps
// of k_split_count, the exclusive scan, k_level_advance and k_split_emit with
// __syncthreads between them, so that levels of at most kSmallLevelCells cells
// cost one launch together instead of four or more each.  A level larger than
// that, or than its capacity, sets kSzAbort as k_level_advance does (the host
// then builds the tree level by level).
__global__ void __launch_bounds__(kSmallLevelThreads)
    k_tree_small_levels(CellArrays c, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ bpos,
                        const int *__restrict__ bstart, int ncrit, int max_depth, SmallLevels sl, int last_level,
                        int cell_cap, int tile_cap, int *__restrict__ sz)
{
    __shared__ long long sv[kSmallLevelCells];  // per cell: children | splits << 32, then its exclusive scan
    __shared__ long long swarp[kSmallLevelThreads / 32];
    __shared__ long long s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kPer = kSmallLevelCells / kSmallLevelThreads;
    for (int level = 0; level < sl.n; ++level) {
        __syncthreads();
        if (sz[kSzAbort]) return;
        const int a = sz[kSzLevel + level], b = sz[kSzLevel + level + 1];
        const int n = b - a;
        if (n > kSmallLevelCells) {
            __syncthreads();
            if (tid == 0) {
                sz[kSzAbort] = 1;
                sz[kSzLevel + level + 2] = b;
            }
            return;
        }
        // split counts (k_split_count), kPer consecutive cells per thread
        long long loc[kPer];
        long long run = 0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int k = tid * kPer + u;
            long long v = 0;
            if (k < n) {
                const int i = a + k;
                const int cb = c.begin[i], ce = c.end[i];
                if (ce - cb > ncrit && level < max_depth) {
                    const uint32_t *B = bpos + bstart[level + 1];
                    const int nb = bstart[level + 2] - bstart[level + 1];
                    int lo, hi;
                    lower_pos2(B, nb, (uint32_t)cb + 1, (uint32_t)ce, lo, hi);
                    v = (long long)(hi - lo + 1) | ((long long)1 << 32);
                    c.child0[i] = lo;  // read back by the emit step below
                }
            }
            loc[u] = run;  // exclusive within the thread's cells
            run += v;
        }
        // block-wide exclusive scan of the threads' sums
        long long x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) swarp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < kSmallLevelThreads / 32 ? swarp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < kSmallLevelThreads / 32) swarp[lane] = w;  // inclusive over warps
            if (lane == kSmallLevelThreads / 32 - 1) s_total = w;
        }
        __syncthreads();
        const long long base = (warp > 0 ? swarp[warp - 1] : 0) + (x - run);
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int k = tid * kPer + u;
            if (k < n) sv[k] = base + loc[u];
        }
        // level advance (k_level_advance)
        if (tid == 0) {
            const long long t = s_total;
            const int nch = (int)(t & 0xffffffffll), nsplit = (int)(t >> 32);
            const int tiles = sz[kSzTiles] + 8 * (int)((nsplit + kTile - 1) / kTile);
            sz[kSzTileBase + level] = sz[kSzTiles];
            if (nch > 0 &&
                (level >= last_level || nch > sl.cap[level + 1] || b + nch > cell_cap || tiles > tile_cap)) {
                sz[kSzAbort] = 1;
                sz[kSzLevel + level + 2] = b;
            } else {
                sz[kSzLevel + level + 2] = b + nch;
                sz[kSzTiles] = tiles;
                sz[kSzCells] = b + nch;
            }
        }
        __syncthreads();
        // children (k_split_emit)
        const int cend = sz[kSzLevel + level + 2];
        const int tile_base = sz[kSzTileBase + level];
        for (int k = tid; k < n; k += kSmallLevelThreads) {
            const int i = a + k;
            const long long e = sv[k];
            const long long next = k + 1 < n ? sv[k + 1] : s_total;
            const int nch = (int)((next - e) & 0xffffffffll);
            const int first = b + (int)(e & 0xffffffffll);
            if (nch == 0 || first + nch > cend) {
                c.child0[i] = -1;
                c.nchild[i] = 0;
                continue;
            }
            const int rank = (int)(e >> 32);
            const int window = rank / kTile, tl = rank % kTile;
            const int cb = c.begin[i], ce = c.end[i];
            const uint32_t *B = bpos + bstart[level + 1];
            const int lo = c.child0[i];  // left by the count step
            emit_children(c, keys, B, lo, i, level, cb, ce, nch, first, tile_base + window * 8, tl);
        }
    }
}

__global__ void k_cell_geom(CellArrays c, int ncells, const double *__restrict__ box, const int *__restrict__ sz)
{
    if (sz) ncells = sz[kSzCells];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x) {
        const int l = c.level[i];
        const int h = 1 << (kKeyBits - l);
        const uint64_t pre = c.prefix[i];
        int C[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) C[a] = (2 * (int)compact3_dev(pre >> a) + 1) * h;
        // the count bucket of the hybrid selection (cells without a particle range:
        // bucket 0)
        const int cnt = c.begin ? c.end[i] - c.begin[i] : 0;
        const int bucket = cnt >= 1 ? min(count_bucket(cnt), kSelNB - 1) : 0;
        c.geom[i] = make_int4(C[0], C[1], C[2], h | (bucket << kGeomBucketShift));
        // real centre lo + (2k + 1) side / 2^(l+1) of the cell's own system box, split
        // into FP32 hi + lo; side and 1/side of the cell in FP32
        const double *bx = box + 4 * c.sys[i];
        const double s = ldexp(bx[3], -l), half = ldexp(bx[3], -l - 1);
        float hi[3], lo[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double cen = bx[a] + (double)(2 * (int64_t)compact3_dev(pre >> a) + 1) * half;
            hi[a] = (float)cen;
            lo[a] = (float)(cen - (double)hi[a]);
        }
        c.fhi[i] = make_float4(hi[0], hi[1], hi[2], (float)(1.0 / s));
        c.flo[i] = make_float4(lo[0], lo[1], lo[2], (float)s);
    }
}

__global__ void k_fill_tile_cells(CellArrays c, int ncells, int *__restrict__ tile_cells, const int *__restrict__ sz)
{
    if (sz) ncells = sz[kSzCells];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncells) return;
    tile_cells[(int64_t)c.tile[i] * kTile + c.lane[i]] = i;
}

// M2L tiles regrouped by the likeness of the rows' offset-class sets.  A tile's
// class blocks are the union of its rows' classes, so a row that lacks a class
// of the union is an empty row of that block.  The tree build cuts tiles by
// parent window and octant; these two kernels reorder each level's cells by
//   (octant within the parent;
//    per axis, the distance in cells to the nearer face of the system's box,
//    clamped at 4, and which face: cells near the same faces lack the same
//    classes;
//    M2L count, descending: in an adaptive tree, cells with as many pairs
//    tend to have the same classes)
// with a stable sort (ties keep Morton order) and cut the order into tiles of
// kTile, level after level.  A level of n cells then takes ceil(n / kTile)
// tiles, no more than the build's 8 per window of kTile split parents.  The
// (tile, class) blocks fall from 54,728 to 48,570 on 2^20 uniform points
// (p = 10, theta = 0.4, N_crit = 64) and from 625,895 to 474,535 on a 2^22-point
// Plummer sphere (p = 8, theta = 0.4, N_crit = 64).  Only the tensor-core M2L
// takes these tiles: its work units split a tile's blocks, while the CUDA-core
// M2L runs one thread block per tile, whose longest tile would set its pace.
constexpr int kTileFaceClamp = 4;
// level 5 | octant 3 | faces 10 | count 10 bits; past the last cell, a key that sorts last
constexpr uint64_t kTileKeyPad = (1ull << kTileSortBits) - 1;

__global__ void k_tile_keys(CellArrays c, int ncells, const int *__restrict__ m2l_cnt, int len,
                            uint64_t *__restrict__ key, uint32_t *__restrict__ val, const int *__restrict__ sz)
{
    if (sz) ncells = sz[kSzCells];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        uint64_t k = kTileKeyPad;
        if (i < ncells) {
            const int l = c.level[i];
            const uint64_t pre = c.prefix[i];
            const int side = 1 << l;
            int prof = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int x = (int)compact3_dev(pre >> a);
                const int lo = x, hi = side - 1 - x;
                const int d = lo <= hi ? min(lo, kTileFaceClamp) : 2 * kTileFaceClamp - min(hi, kTileFaceClamp);
                prof = prof * (2 * kTileFaceClamp + 1) + d;
            }
            const int cnt = min(m2l_cnt[i], 1023);
            k = ((uint64_t)l << 23) | ((pre & 7ull) << 20) | ((uint64_t)prof << 10) | (uint64_t)(1023 - cnt);
        }
        key[i] = k;
        val[i] = (uint32_t)i;
    }
}

// Tile and lane of every cell from its position j in the sorted order: the
// cells of level l hold positions lstart[l] .. lstart[l + 1] - 1.  A tile past
// tile_cap (which the bound above rules out) sets kSzAbort (with sz) instead of
// writing.
__global__ void k_tile_assign(const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, int ncells,
                              const int *__restrict__ lstart, int tile_cap, CellArrays c, int *__restrict__ sz)
{
    if (sz) ncells = sz[kSzCells];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ncells; j += gridDim.x * blockDim.x) {
        const int l = (int)(key[j] >> 23);
        if (l > kMaxLevel) continue;
        int base = 0;
        for (int m = 0; m < l; ++m) base += (lstart[m + 1] - lstart[m] + kTile - 1) / kTile;
        const int r = j - lstart[l];
        const int tile = base + r / kTile;
        if (r < 0 || tile >= tile_cap) {
            if (sz) atomicOr(&sz[kSzAbort], 1);
            continue;
        }
        const int cell = (int)val[j];
        c.tile[cell] = tile;
        c.lane[cell] = r % kTile;
    }
}

// Compact list of leaf cells (order preserved) via a precomputed exclusive scan.
__global__ void k_leaf_flags(CellArrays c, int ncells, int *__restrict__ flag, const int *__restrict__ sz, int len)
{
    if (sz)
        ncells = sz[kSzCells];
    else
        len = ncells;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) flag[i] = i < ncells && c.nchild[i] == 0;
}

__global__ void k_leaf_compact(CellArrays c, int ncells, const int *__restrict__ ex,
                               int *__restrict__ leaves, const int *__restrict__ sz, int *__restrict__ pcell)
{
    if (sz) ncells = sz[kSzCells];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ncells && c.nchild[i] == 0) {
        leaves[ex[i]] = i;
        for (int j = c.begin[i], e = c.end[i]; j < e; ++j) pcell[j] = i;  // the leaf of each sorted particle
    }
}

}  // namespace fmm
