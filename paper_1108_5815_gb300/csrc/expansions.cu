// expansions.cu -- spherical-harmonic expansions on the GPU: operator tables
// (FP64 -> FP32), P2M, M2M, L2L and L2P (FP32).
//
// The paper's kernels are "based on spherical harmonic expansions" of order p
// (section "Hybrid treecode/FMM algorithm").  With the solid harmonics
//   R_n^m(x) = r^n P_n^m(cos t) e^{imf} / (n+m)!,
//   I_n^m(x) = (n-m)! P_n^m(cos t) e^{imf} / r^{n+1},
// 1/|x-y| = sum conj(R_n^m(y)) I_n^m(x) and the operators are
//   P2M  M_n^m  = sum q conj(R_n^m(y - c))
//   M2M  M'_n^m = sum conj(R_k^l(c - c')) M_{n-k}^{m-l}
//   M2L  L_j^l  = (-1)^{j+l} sum M_n^m I_{n+j}^{m-l}(c_t - c_s)
//   L2L  L'_j^l = sum L_n^m R_{n-j}^{m-l}(c' - c)
//   L2P  phi = sum L_n^m R_n^m(x - c), (d/dz) phi = sum L_n^m R_{n-1}^m,
//        (d/dx + i d/dy) phi = sum L_n^m R_{n-1}^{m+1}.
// Storage on the GPU (documented in fmm.h): m >= 0 only, real layout
// [Re c_n^0, Re c_n^1, Im c_n^1, ...] per degree, each cell's row padded to
// P2pad floats, and two rescalings that keep every quantity O(1) in FP32:
//   * unit scaling by the cell side s: M~_n = M_n s^-n, L~_j = L_j s^{j+1},
//     which makes every operator matrix independent of the level;
//   * the order normalisation nu_n^m = sqrt((n-m)!(n+m)!):
//     M^_n^m = nu_n^m M~_n^m and L^_n^m = L~_n^m / nu_n^m, i.e. the expansions
//     are taken in the basis R^ = nu R, whose recurrence
//       R^_m^m = -(x+iy) sqrt((2m-1)/(2m)) R^_{m-1}^{m-1}
//       R^_n^m = ((2n-1) z R^_{n-1}^m - r^2 sqrt((n-m-1)(n+m-1)) R^_{n-2}^m)
//                / sqrt((n+m)(n-m))
//     stays bounded by |x|^n.
// The M2L/M2M/L2L operators become real (P2 x P2) matrices, computed in FP64
// from the complex formulas and stored in FP32.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

struct cd {
    double re, im;
};

__device__ __forceinline__ cd cmul(cd a, cd b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

__device__ __forceinline__ int tri(int n, int m) { return n * (n + 1) / 2 + m; }

// log-free sqrt((n-m)!(n+m)!) in FP64 (n <= 40).
__device__ double nu(int n, int m)
{
    m = m < 0 ? -m : m;
    double f = 1.0;
    for (int k = 2; k <= n - m; ++k) f *= k;
    for (int k = 2; k <= n + m; ++k) f *= k;
    return sqrt(f);
}

// Plain (un-normalised) regular harmonics R_n^m, m >= 0, n <= P, in FP64.
__device__ void regular_fp64(double x, double y, double z, int P, cd *R)
{
    const double r2 = x * x + y * y + z * z;
    for (int m = 0; m <= P; ++m) {
        cd rmm;
        if (m == 0) {
            rmm = {1.0, 0.0};
        } else {
            const cd prev = R[tri(m - 1, m - 1)];
            const cd u = {-x / (2.0 * m), -y / (2.0 * m)};
            rmm = cmul(u, prev);
        }
        R[tri(m, m)] = rmm;
        cd p2 = {0.0, 0.0}, p1 = rmm;
        for (int n = m + 1; n <= P; ++n) {
            const double inv = 1.0 / ((double)(n + m) * (double)(n - m));
            cd rn = {((2.0 * n - 1.0) * z * p1.re - r2 * p2.re) * inv,
                     ((2.0 * n - 1.0) * z * p1.im - r2 * p2.im) * inv};
            R[tri(n, m)] = rn;
            p2 = p1;
            p1 = rn;
        }
    }
}

// Plain irregular harmonics I_n^m, m >= 0, n <= P, in FP64.
__device__ void irregular_fp64(double x, double y, double z, int P, cd *Ih)
{
    const double r2 = x * x + y * y + z * z;
    const double ir2 = 1.0 / r2;
    for (int m = 0; m <= P; ++m) {
        cd imm;
        if (m == 0) {
            imm = {1.0 / sqrt(r2), 0.0};
        } else {
            const cd prev = Ih[tri(m - 1, m - 1)];
            const double f = -(2.0 * m - 1.0) * ir2;
            imm = cmul({f * x, f * y}, prev);
        }
        Ih[tri(m, m)] = imm;
        cd p2 = {0.0, 0.0}, p1 = imm;
        for (int n = m + 1; n <= P; ++n) {
            const double a = (2.0 * n - 1.0) * z, b = (double)(n + m - 1) * (double)(n - m - 1);
            cd in = {(a * p1.re - b * p2.re) * ir2, (a * p1.im - b * p2.im) * ir2};
            Ih[tri(n, m)] = in;
            p2 = p1;
            p1 = in;
        }
    }
}

// Signed-m access to a harmonic table with H_n^{-m} = (-1)^m conj(H_n^m).
__device__ __forceinline__ cd hsigned(const cd *H, int n, int m)
{
    if (m >= 0) return H[tri(n, m)];
    const cd v = H[tri(n, -m)];
    return (m & 1) ? cd{-v.re, v.im} : cd{v.re, -v.im};
}


enum { kOpM2L = 0, kOpM2M = 1, kOpL2L = 2 };

// Complex coefficient of input coefficient (n, m) [signed m] in output (j, l)
// [l >= 0], in the normalised unit-scaled basis.
__device__ cd op_coef(int op, const cd *H, int j, int l, int n, int m, double rho, int p)
{
    if (op == kOpM2L) {
        // L_j^l = (-1)^{j+l} rho^n sum M_n^m I_{n+j}^{m-l}
        const cd v = hsigned(H, n + j, m - l);
        double f = (((j + l) & 1) ? -1.0 : 1.0) * pow(rho, (double)n) / (nu(j, l) * nu(n, m));
        return {v.re * f, v.im * f};
    }
    if (op == kOpM2M) {
        // M'_j^l = sum conj(R_k^d) 2^{-n} M_n^m, k = j - n, d = l - m
        const int k = j - n, d = l - m;
        if (k < 0 || (d < 0 ? -d : d) > k) return {0.0, 0.0};
        const cd v = hsigned(H, k, d);
        const double f = ldexp(1.0, -n) * nu(j, l) / nu(n, m);
        return {v.re * f, -v.im * f};
    }
    // L2L: L'_j^l = sum 2^{-n-1} R_{n-j}^{m-l} L_n^m
    const int k = n - j, d = m - l;
    if (k < 0 || (d < 0 ? -d : d) > k) return {0.0, 0.0};
    const cd v = hsigned(H, k, d);
    const double f = ldexp(1.0, -n - 1) * nu(n, m) / nu(j, l);
    return {v.re * f, v.im * f};
}

// Real matrix entry: output real index `row` <- input real index `col`.
__device__ double real_entry(int op, const cd *H, int row, int col, double rho, int p)
{
    int j = 0;
    while ((j + 1) * (j + 1) <= row) ++j;
    int rr = row - j * j;
    const int l = (rr + 1) / 2;
    const int rim = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
    int n = 0;
    while ((n + 1) * (n + 1) <= col) ++n;
    int cc = col - n * n;
    const int mm = (cc + 1) / 2;
    const int cim = (cc == 0) ? 0 : ((cc & 1) ? 0 : 1);
    const cd A = op_coef(op, H, j, l, n, mm, rho, p);
    cd B = {0.0, 0.0};
    if (mm > 0) {
        const cd b = op_coef(op, H, j, l, n, -mm, rho, p);
        const double s = (mm & 1) ? -1.0 : 1.0;
        B = {b.re * s, b.im * s};
    }
    if (rim == 0) return cim == 0 ? A.re + B.re : -A.im + B.im;
    return cim == 0 ? A.im + B.im : A.re - B.re;
}

}  // namespace

// One block per new offset class: decode (dl, d), compute I^(delta) in FP64
// and write the P2pad x P2pad matrix (row = output, col = input) at its cache slot.
__global__ void k_build_m2l_tables(const uint64_t *__restrict__ class_keys,
                                   const int *__restrict__ cache_slot, int nnew, int p, int P2pad,
                                   float *__restrict__ table)
{
    extern __shared__ cd sh_h[];
    const int ci = blockIdx.x;
    if (ci >= nnew) return;
    const uint64_t key = class_keys[ci];
    const int dl = (int)(key >> 57) - 64;  // level(S) - level(T)
    int64_t d[3];
    for (int a = 0; a < 3; ++a) d[a] = (int64_t)((key >> (38 - 19 * a)) & 0x7ffff) - (1 << 18);
    // delta = d / s_T and rho = s_S / s_T, both powers of two times d
    const int fine_shift = dl >= 0 ? dl + 1 : 1;
    const double rho = ldexp(1.0, -dl);
    const double dx = ldexp((double)d[0], -fine_shift), dy = ldexp((double)d[1], -fine_shift),
                 dz = ldexp((double)d[2], -fine_shift);
    if (threadIdx.x == 0) irregular_fp64(dx, dy, dz, 2 * p, sh_h);
    __syncthreads();
    const int P2 = nterms(p);
    float *out = table + (int64_t)cache_slot[ci] * P2pad * P2pad;
    for (int e = threadIdx.x; e < P2pad * P2pad; e += blockDim.x) {
        const int row = e / P2pad, col = e % P2pad;
        double v = 0.0;
        if (row < P2 && col < P2) v = real_entry(kOpM2L, sh_h, row, col, rho, p);
        out[e] = (float)v;
    }
}

// Blocks 0..7: M2M matrices per child octant; blocks 8..15: L2L.  Stored
// transposed (input-major): t[o][col][row] so that consecutive threads (rows)
// read consecutive addresses.
__global__ void k_build_shift_tables(int p, int P2pad, float *__restrict__ m2m,
                                     float *__restrict__ l2l, double *__restrict__ m2m64,
                                     double *__restrict__ l2l64)
{
    extern __shared__ cd sh_h[];
    const int op = blockIdx.x < 8 ? kOpM2M : kOpL2L;
    const int o = blockIdx.x & 7;
    const double sgn[3] = {(o & 1) ? 1.0 : -1.0, (o & 2) ? 1.0 : -1.0, (o & 4) ? 1.0 : -1.0};
    // M2M: (child - parent) / parent side = +-1/4; L2L: (child - parent) / child side = +-1/2
    const double f = op == kOpM2M ? 0.25 : 0.5;
    if (threadIdx.x == 0) regular_fp64(sgn[0] * f, sgn[1] * f, sgn[2] * f, p, sh_h);
    __syncthreads();
    const int P2 = nterms(p);
    float *out = (op == kOpM2M ? m2m : l2l) + (int64_t)o * P2pad * P2pad;
    double *out64 = op == kOpM2M ? m2m64 : l2l64;
    if (out64) out64 += (int64_t)o * P2pad * P2pad;
    for (int e = threadIdx.x; e < P2pad * P2pad; e += blockDim.x) {
        const int col = e / P2pad, row = e % P2pad;
        double v = 0.0;
        if (row < P2 && col < P2) v = real_entry(op, sh_h, row, col, 1.0, p);
        out[e] = (float)v;
        if (out64) out64[e] = v;
    }
}

// ---------------------------------------------------------------- P2M / L2P

namespace {

__device__ __forceinline__ void cell_centre_side(const CellArrays &c, int cell,
                                                 const double *__restrict__ box, double cen[3],
                                                 double &s)
{
    const int l = c.level[cell];
    const uint64_t pre = c.prefix[cell];
    const double *bx = box + 4 * c.sys[cell];  // the box of the cell's own system
    s = ldexp(bx[3], -l);
    const double half = ldexp(bx[3], -l - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) cen[a] = bx[a] + (double)(2 * (int64_t)compact3_dev(pre >> a) + 1) * half;
}

constexpr int kMaxChunks = 14;  // ceil(448 / 32): p <= 20

// A particle's offset from a cell's centre in units of the cell side, in FP32:
// ((x - c_hi) - c_lo) / s with the centre's FP32 hi + lo parts (k_cell_geom).
struct Frame {
    float4 hi, lo;
};
__device__ __forceinline__ Frame cell_frame(const CellArrays &c, int cell) { return {c.fhi[cell], c.flo[cell]}; }
__device__ __forceinline__ void frame_offset(const Frame &f, float4 pt, float &x, float &y, float &z)
{
    x = __fmul_rn(__fsub_rn(__fsub_rn(pt.x, f.hi.x), f.lo.x), f.hi.w);
    y = __fmul_rn(__fsub_rn(__fsub_rn(pt.y, f.hi.y), f.lo.y), f.hi.w);
    z = __fmul_rn(__fsub_rn(__fsub_rn(pt.z, f.hi.z), f.lo.z), f.hi.w);
}

}  // namespace

// Coefficients of the order-normalised three-term recurrences, for n <= kRecMax
// at index n(n+1)/2 + m:  R^_n^m = kRecA z R^_{n-1}^m - kRecB r^2 R^_{n-2}^m and
// I^_n^m = (kRecA z I^_{n-1}^m - kRecB I^_{n-2}^m) / r^2, with
// kRecA = (2n-1)/sqrt((n+m)(n-m)), kRecB = sqrt((n+m-1)(n-m-1))/sqrt((n+m)(n-m));
// diagonals R^_m^m = kRecD (x+iy) R^_{m-1}^{m-1} (I^ likewise over r^2),
// kRecD = -sqrt((2m-1)/(2m)).  Filled once per device from FP64 values.
constexpr int kRecMax = 21;
constexpr int kRecTri = (kRecMax + 1) * (kRecMax + 2) / 2;
__constant__ float c_rec_a[kRecTri], c_rec_b[kRecTri], c_rec_d[kRecMax + 1];
// L2P derivative weights per stored coefficient index k (n, m from k):
// sqrt((n-m)(n+m)), sqrt((n-m)(n-m-1)), sqrt((n+m)(n+m-1)); global memory, since
// the lanes of a warp read different entries.
constexpr int kScaleMax = 448;
__device__ float g_l2p_scale[3][kScaleMax];
// P2M writes the real coefficients of a particle in the order its recurrences
// produce them (orders m and m + 1 together: (m, m), then (n, m), (n, m + 1)
// for n = m + 1..p, a term m > 0 giving its real and imaginary parts); entry
// [p][g] is the stored coefficient index of the g-th value produced.
__device__ short g_p2m_perm[kRecMax][kScaleMax];

void init_recurrence_tables()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && done[dev]) return;
    float a[kRecTri], b[kRecTri], d[kRecMax + 1];
    for (int n = 0; n <= kRecMax; ++n)
        for (int m = 0; m <= n; ++m) {
            const int t = n * (n + 1) / 2 + m;
            const double den = n > m ? 1.0 / std::sqrt((double)(n + m) * (n - m)) : 0.0;
            a[t] = (float)((2.0 * n - 1.0) * den);
            b[t] = n > m + 1 ? (float)(std::sqrt((double)(n + m - 1) * (n - m - 1)) * den) : 0.f;
        }
    for (int m = 0; m <= kRecMax; ++m) d[m] = m > 0 ? (float)-std::sqrt((2.0 * m - 1.0) / (2.0 * m)) : 1.f;
    static float sc[3][kScaleMax];
    for (int k = 0; k < kScaleMax; ++k) {
        int n = 0;
        while ((n + 1) * (n + 1) <= k) ++n;
        const int m = (k - n * n + 1) / 2;
        sc[0][k] = (float)std::sqrt((double)(n - m) * (n + m));
        sc[1][k] = (float)std::sqrt((double)std::max(0, (n - m) * (n - m - 1)));
        sc[2][k] = (float)std::sqrt((double)(n + m) * (n + m - 1));
    }
    FMM_CUDA_TRY(cudaMemcpyToSymbol(g_l2p_scale, sc, sizeof(sc)));
    static short perm[kRecMax][kScaleMax];
    for (int pp = 0; pp < kRecMax; ++pp) {
        int g = 0;
        auto put = [&](int n, int m) {
            if (m == 0) {
                perm[pp][g++] = (short)(n * n);
            } else {
                perm[pp][g++] = (short)(n * n + 2 * m - 1);
                perm[pp][g++] = (short)(n * n + 2 * m);
            }
        };
        for (int m = 0; m <= pp; m += 2) {
            put(m, m);
            for (int n = m + 1; n <= pp; ++n) {
                put(n, m);
                put(n, m + 1);
            }
        }
        for (; g < kScaleMax; ++g) perm[pp][g] = -1;
    }
    FMM_CUDA_TRY(cudaMemcpyToSymbol(g_p2m_perm, perm, sizeof(perm)));
    FMM_CUDA_TRY(cudaMemcpyToSymbol(c_rec_a, a, sizeof(a)));
    FMM_CUDA_TRY(cudaMemcpyToSymbol(c_rec_b, b, sizeof(b)));
    FMM_CUDA_TRY(cudaMemcpyToSymbol(c_rec_d, d, sizeof(d)));
    if (dev < 64) done[dev] = true;
}

// One warp per leaf.  Each lane evaluates q R^(x - c) of one particle; the
// values are written, in the order the recurrences produce them, into a 32 x 32
// tile of shared memory (a row per lane), and every 32 values the lanes sum the
// tile's columns, so a warp needs only 6 KB of shared memory.  The column sums
// accumulate per produced value in shared memory and are written to their
// stored indices at the end.
// PT > 0: the expansion order as a compile-time constant (loops unrolled, the
// recurrence coefficients and shared-memory offsets folded); PT = 0: p at run time.
template <int PT>
__global__ void __launch_bounds__(32)
    k_p2m(CellArrays c, const int *__restrict__ leaves, int nleaves, const float4 *__restrict__ pts,
          int p_run, int P2pad, float *__restrict__ M, const int *__restrict__ sz)
{
    const int p = PT > 0 ? PT : p_run;
    __shared__ float tile[32 * 33];
    __shared__ float colsum[kMaxChunks * 32];  // sums of produced values, by batch of 32
    if (sz) nleaves = sz[kSzLeaves];
    const int li = blockIdx.x;
    if (li >= nleaves) return;
    const int cell = leaves[li];
    const int lane = threadIdx.x;
    const Frame fr = cell_frame(c, cell);
    const int b = c.begin[cell], e = c.end[cell];
    const int P2 = nterms(p);
    for (int j = lane; j < kMaxChunks * 32; j += 32) colsum[j] = 0.f;
    float *row = tile + lane * 33;
    for (int base = b; base < e; base += 32) {
        const int i = base + lane;
        // a lane past the leaf's end adds zeros: charge 0 at the centre (finite harmonics)
        float x = 0.f, y = 0.f, z = 0.f, q = 0.f;
        if (i < e) {
            const float4 pt = pts[i];
            frame_offset(fr, pt, x, y, z);
            q = pt.w;
        }
        const float r2 = x * x + y * y + z * z;
        int g = 0;  // values produced so far (the same in every lane)
        auto flush = [&]() {
            __syncwarp();
            float sum = 0.f;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) sum += tile[r * 33 + lane];
            colsum[((g - 1) & ~31) + lane] += sum;
            __syncwarp();
        };
        auto put1 = [&](float v) {
            row[g & 31] = v;
            if ((++g & 31) == 0) flush();
        };
        auto put = [&](int m, float rr, float ri) {
            put1(q * rr);
            if (m > 0) put1(-q * ri);
        };
        // orders m and m + 1 advance together: two independent recurrences in n
        float mre = 1.f, mim = 0.f;  // R^_m^m
#pragma unroll
        for (int m = 0; m <= p; m += 2) {
            if (m > 0) {
                const float f = c_rec_d[m];
                const float nre = f * (x * mre - y * mim), nim = f * (x * mim + y * mre);
                mre = nre;
                mim = nim;
            }
            float bre = 0.f, bim = 0.f;  // R^_{m+1}^{m+1}
            if (m + 1 <= p) {
                const float f = c_rec_d[m + 1];
                bre = f * (x * mre - y * mim);
                bim = f * (x * mim + y * mre);
            }
            put(m, mre, mim);
            float a2r = 0.f, a2i = 0.f, a1r = mre, a1i = mim;  // chain m
            float b2r = 0.f, b2i = 0.f, b1r = bre, b1i = bim;  // chain m + 1
#pragma unroll
            for (int n = m + 1; n <= p; ++n) {
                const int ta = n * (n + 1) / 2 + m;
                const float aa = c_rec_a[ta] * z, ab = c_rec_b[ta] * r2;
                const float rr = aa * a1r - ab * a2r, ri = aa * a1i - ab * a2i;
                a2r = a1r;
                a2i = a1i;
                a1r = rr;
                a1i = ri;
                put(m, rr, ri);
                float qr = b1r, qi = b1i;  // n == m + 1: the diagonal itself
                if (n > m + 1) {
                    const int tb = ta + 1;
                    const float ba = c_rec_a[tb] * z, bb = c_rec_b[tb] * r2;
                    qr = ba * b1r - bb * b2r;
                    qi = ba * b1i - bb * b2i;
                    b2r = b1r;
                    b2i = b1i;
                    b1r = qr;
                    b1i = qi;
                }
                put(m + 1, qr, qi);
            }
            mre = bre;  // the next pair starts from R^_{m+1}^{m+1}
            mim = bim;
        }
        if (g & 31) {  // the last, partial tile: zero its unused columns first
            for (int k = g & 31; k < 32; ++k) row[k] = 0.f;
            g = (g | 31) + 1;
            flush();
        }
    }
    __syncwarp();
    float *out = M + (int64_t)cell * P2pad;
    for (int gg = lane; gg < P2; gg += 32) out[g_p2m_perm[p][gg]] = colsum[gg];
    for (int k = P2 + lane; k < P2pad; k += 32) out[k] = 0.f;
}

void launch_p2m(const CellArrays &c, const int *leaves, int nleaves, unsigned grid, const float4 *pts, int p,
                int P2pad, float *M, cudaStream_t st, const int *sz)
{
    switch (p) {
#define FMM_P2M_CASE(P)                                                            \
    case P:                                                                        \
        k_p2m<P><<<grid, 32, 0, st>>>(c, leaves, nleaves, pts, p, P2pad, M, sz); \
        break;
        FMM_P2M_CASE(4)
        FMM_P2M_CASE(6)
        FMM_P2M_CASE(8)
        FMM_P2M_CASE(10)
        FMM_P2M_CASE(12)
#undef FMM_P2M_CASE
    default:
        k_p2m<0><<<grid, 32, 0, st>>>(c, leaves, nleaves, pts, p, P2pad, M, sz);
    }
    FMM_LAUNCH_CHECK();
}

// Octant-batched shifts.  A block takes 32 consecutive parents of one level, one
// octant o and one 128-row tile of output coefficients, and multiplies the
// octant's matrix (read once per block, 32 K-rows at a time through shared
// memory) with the rows of the 32 (parent, child with octant o) pairs at once:
//   M2M: T_child = A_o M^_child   (then M^_parent = sum of T over its children,
//        in octant order, k_m2m_sum);
//   L2L: L^_child += A_o L^_parent.
// A matrix is column-major: entry (row j, column k) at k * P2pad + j.  Each
// thread keeps 4 output rows x 8 pairs in registers.
template <bool L2L>
__global__ void __launch_bounds__(128)
    k_shift_batched(CellArrays c, int a, int b, const float *__restrict__ mats, int P2, int P2pad,
                    const float *in, float *out,  // L2L: in and out are the same array (disjoint rows)
                    const int *__restrict__ sz, int level)
{
    __shared__ __align__(16) float sA[32][128];
    __shared__ __align__(16) float sC[32][32];
    __shared__ int sch[32];
    __shared__ int sany;
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
    }
    const int t = threadIdx.x;
    const int p0 = a + blockIdx.x * 32;
    const int np = min(32, b - p0);
    const int j0 = blockIdx.y * 128;
    const int o = blockIdx.z;
    const int jg = t & 31, pg = t >> 5;  // rows j0 + 4 jg .. +3, pairs 8 pg .. +7
    if (t == 0) sany = 0;
    __syncthreads();
    if (t < 32) {
        int ch = -1;
        if (t < np) {
            const int P = p0 + t, c0 = c.child0[P], nch = c.nchild[P];
            for (int k = 0; k < nch; ++k)
                if ((int)(c.prefix[c0 + k] & 7ull) == o) ch = c0 + k;
        }
        sch[t] = ch;
        if (ch >= 0) sany = 1;
    }
    __syncthreads();
    if (!sany) return;
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
    const float *A = mats + (int64_t)o * P2pad * P2pad;
    // The next K-chunk is loaded into registers (all loads of a thread in flight
    // at once) while the current one is multiplied: one memory latency per chunk
    // instead of one per element, which is what the small top levels wait on.
    // A chunk: 32 K-rows x 128 output rows of A (8 float4 per thread) and 32 K
    // entries of the 32 input rows (2 float4 per thread, parent q = idx & 31).
    // P2pad is a multiple of 32, so every float4 is aligned and inside its row.
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ra[8], rc[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = t + 128 * i;
            const int kr = idx >> 5, jj = (idx & 31) * 4;
            const int k = k0 + kr, j = j0 + jj;
            ra[i] = (k < P2 && j < P2pad) ? __ldg(reinterpret_cast<const float4 *>(A + (int64_t)k * P2pad + j)) : zero4;
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int idx = t + 128 * i;
            const int q = idx & 31, k = k0 + (idx >> 5) * 4;
            const int row = L2L ? (sch[q] >= 0 ? p0 + q : -1) : sch[q];
            float4 v = zero4;
            if (row >= 0 && k < P2) {
                v = *reinterpret_cast<const float4 *>(in + (int64_t)row * P2pad + k);
                if (k + 1 >= P2) v.y = 0.f;
                if (k + 2 >= P2) v.z = 0.f;
                if (k + 3 >= P2) v.w = 0.f;
            }
            rc[i] = v;
        }
    };
    load(0);
    for (int k0 = 0; k0 < P2; k0 += 32) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = t + 128 * i;
            *reinterpret_cast<float4 *>(&sA[idx >> 5][(idx & 31) * 4]) = ra[i];
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int idx = t + 128 * i;
            const int q = idx & 31, kr = (idx >> 5) * 4;
            sC[kr][q] = rc[i].x;
            sC[kr + 1][q] = rc[i].y;
            sC[kr + 2][q] = rc[i].z;
            sC[kr + 3][q] = rc[i].w;
        }
        __syncthreads();
        if (k0 + 32 < P2) load(k0 + 32);
#pragma unroll 8
        for (int kr = 0; kr < 32; ++kr) {
            const float4 av = *reinterpret_cast<const float4 *>(&sA[kr][4 * jg]);
            const float4 c0v = *reinterpret_cast<const float4 *>(&sC[kr][8 * pg]);
            const float4 c1v = *reinterpret_cast<const float4 *>(&sC[kr][8 * pg + 4]);
            const float aa[4] = {av.x, av.y, av.z, av.w};
            const float cc[8] = {c0v.x, c0v.y, c0v.z, c0v.w, c1v.x, c1v.y, c1v.z, c1v.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(aa[r], cc[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ch = sch[8 * pg + q];
        if (ch < 0) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = j0 + 4 * jg + r;
            if (j >= P2pad) continue;
            if (L2L) {
                if (j < P2) out[(int64_t)ch * P2pad + j] += acc[r][q];
            } else {
                out[(int64_t)ch * P2pad + j] = j < P2 ? acc[r][q] : 0.f;
            }
        }
    }
}

// M^_parent = sum over its children (octant order) of T_child, parents [a, b).
__global__ void k_m2m_sum(CellArrays c, int a, int b, int P2pad, const float *__restrict__ T, float *__restrict__ M,
                          const int *__restrict__ sz, int level)
{
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
    }
    const int nq = P2pad / 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)(b - a) * nq;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int P = a + (int)(i / nq), q4 = (int)(i % nq);
        const int nch = c.nchild[P];
        if (nch == 0) continue;
        const int c0 = c.child0[P];
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < nch; ++k) {
            const float4 v = reinterpret_cast<const float4 *>(T + (int64_t)(c0 + k) * P2pad)[q4];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        reinterpret_cast<float4 *>(M + (int64_t)P * P2pad)[q4] = s;
    }
}

// The same shifts with FP64 matrices and FP64 sums (rows stored in FP32), for
// the few top-level parents at high p: one block per parent of [a, b).
template <bool L2L>
__global__ void __launch_bounds__(128)
    k_shift_fp64(CellArrays c, int a, int b, const double *__restrict__ mats, int P2, int P2pad, float *E,
                 const int *__restrict__ sz, int level)
{
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
    }
    extern __shared__ double sx[];  // P2pad
    const int P = a + blockIdx.x;
    if (P >= b) return;
    const int nch = c.nchild[P], c0 = c.child0[P];
    if (nch == 0) return;
    if (!L2L) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < nch; ++k) {
            const int ch = c0 + k, o = (int)(c.prefix[ch] & 7ull);
            __syncthreads();
            for (int i = threadIdx.x; i < P2pad; i += blockDim.x) sx[i] = (double)E[(int64_t)ch * P2pad + i];
            __syncthreads();
            const double *A = mats + (int64_t)o * P2pad * P2pad;
            for (int r = 0; r < 4; ++r) {
                const int j = threadIdx.x + r * blockDim.x;
                if (j < P2)
                    for (int col = 0; col < P2; ++col) acc[r] = fma(A[(int64_t)col * P2pad + j], sx[col], acc[r]);
            }
        }
        for (int r = 0; r < 4; ++r) {
            const int j = threadIdx.x + r * blockDim.x;
            if (j < P2pad) E[(int64_t)P * P2pad + j] = j < P2 ? (float)acc[r] : 0.f;
        }
    } else {
        for (int i = threadIdx.x; i < P2pad; i += blockDim.x) sx[i] = (double)E[(int64_t)P * P2pad + i];
        __syncthreads();
        for (int k = 0; k < nch; ++k) {
            const int ch = c0 + k, o = (int)(c.prefix[ch] & 7ull);
            const double *A = mats + (int64_t)o * P2pad * P2pad;
            for (int j = threadIdx.x; j < P2; j += blockDim.x) {
                double v = 0.0;
                for (int col = 0; col < P2; ++col) v = fma(A[(int64_t)col * P2pad + j], sx[col], v);
                E[(int64_t)ch * P2pad + j] += (float)v;
            }
        }
    }
}

void launch_shift_fp64(bool l2l, const CellArrays &c, int a, int b, const double *mats, int P2, int P2pad, float *E,
                       cudaStream_t st, const int *sz, int level, int cap)
{
    const int np = sz ? cap : b - a;
    if (np <= 0) return;
    if (l2l)
        k_shift_fp64<true><<<np, 128, sizeof(double) * P2pad, st>>>(c, a, b, mats, P2, P2pad, E, sz, level);
    else
        k_shift_fp64<false><<<np, 128, sizeof(double) * P2pad, st>>>(c, a, b, mats, P2, P2pad, E, sz, level);
    FMM_LAUNCH_CHECK();
}

void launch_shift_batched(bool l2l, const CellArrays &c, int a, int b, const float *mats, int P2, int P2pad,
                          float *E, float *T, cudaStream_t st, const int *sz, int level, int cap)
{
    const int np = sz ? cap : b - a;  // parents launched for
    if (np <= 0) return;
    const dim3 grid((unsigned)ceil_div(np, 32), (unsigned)ceil_div(P2pad, 128), 8);
    if (l2l) {
        k_shift_batched<true><<<grid, 128, 0, st>>>(c, a, b, mats, P2, P2pad, E, E, sz, level);
        FMM_LAUNCH_CHECK();
    } else {
        k_shift_batched<false><<<grid, 128, 0, st>>>(c, a, b, mats, P2, P2pad, E, T, sz, level);
        FMM_LAUNCH_CHECK();
        const int64_t n = (int64_t)np * (P2pad / 4);
        k_m2m_sum<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16), 256, 0, st>>>(c, a, b, P2pad, T, E, sz,
                                                                                         level);
        FMM_LAUNCH_CHECK();
    }
}

// Far-field potential and gradient from a leaf's local expansion,
// phi = Re sum L^ R^, d/dz and D+ = d/dx + i d/dy from the derivative ladder.
// Every term (n, m), m >= 0, reads one record of 8 floats from shared memory
// (two 16-byte loads), built once per leaf with the normalisation ratios, the
// weight 2 of the m > 0 real parts and the two D+ contributions already
// combined:
//   [w Lr, w Li, w Lzr, w Lzi, X1r - X2r, X1i - X2i, X1r + X2r, X1i + X2i]
// with Lz = L_{n+1}^m s0, X1 = L_{n+1}^{m-1} s1 (m >= 1), X2 = L_{n+1}^{m+1} s2
// (zero past n + 1 > p), so that
//   phi += w(Lr rr - Li ri),  dz += w(Lzr rr - Lzi ri),
//   dpr += (X1r - X2r) rr - (X1i - X2i) ri,  dpi += (X1r + X2r) ri + (X1i + X2i) rr.

// The records of local expansion Lg (P2 floats) into rec (2 ntri float4),
// staging Lg in Lh; the 32 lanes of the warp share the work.
__device__ __forceinline__ void l2p_records(const float *__restrict__ Lg, int p, float *Lh, float4 *rec, int lane)
{
    const int P2 = nterms(p), ntri = (p + 1) * (p + 2) / 2;
    for (int k = lane; k < P2; k += 32) Lh[k] = Lg[k];
    __syncwarp();
    for (int t = lane; t < ntri; t += 32) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= t) ++n;
        const int m = t - n * (n + 1) / 2;
        const float w = m == 0 ? 1.f : 2.f;
        const int k = n * n + (m == 0 ? 0 : 2 * m - 1);
        float lr = Lh[k], lim = m == 0 ? 0.f : Lh[k + 1];
        float zr = 0.f, zi = 0.f, x1r = 0.f, x1i = 0.f, x2r = 0.f, x2i = 0.f;
        if (n + 1 <= p) {
            const int base = (n + 1) * (n + 1);
            const int kz = base + (m == 0 ? 0 : 2 * m - 1);
            zr = Lh[kz] * g_l2p_scale[0][kz];
            zi = m == 0 ? 0.f : Lh[kz + 1] * g_l2p_scale[0][kz];
            if (m >= 1) {
                const int k1 = base + (m == 1 ? 0 : 2 * (m - 1) - 1);
                x1r = Lh[k1] * g_l2p_scale[1][k1];
                x1i = m == 1 ? 0.f : Lh[k1 + 1] * g_l2p_scale[1][k1];
            }
            const int k2 = base + 2 * (m + 1) - 1;
            x2r = Lh[k2] * g_l2p_scale[2][k2];
            x2i = Lh[k2 + 1] * g_l2p_scale[2][k2];
        }
        rec[2 * t] = make_float4(w * lr, w * lim, w * zr, w * zi);
        rec[2 * t + 1] = make_float4(x1r - x2r, x1i - x2i, x1r + x2r, x1i + x2i);
    }
    __syncwarp();
}

// phi and grad at particle pt from the records of its leaf (frame fr).
template <int PT>
__device__ __forceinline__ float4 l2p_eval(const float4 *rec, const Frame &fr, float4 pt, int p_run)
{
    const int p = PT > 0 ? PT : p_run;
    const float inv_s = fr.hi.w, inv_s2 = inv_s * inv_s;
    struct Sums {
        float phi, dz, dpr, dpi;
    };
    auto term = [&](int t, float rr, float ri, Sums &sm) {
        const float4 u = rec[2 * t], v = rec[2 * t + 1];
        sm.phi = fmaf(u.x, rr, fmaf(-u.y, ri, sm.phi));
        sm.dz = fmaf(u.z, rr, fmaf(-u.w, ri, sm.dz));
        sm.dpr = fmaf(v.x, rr, fmaf(-v.y, ri, sm.dpr));
        sm.dpi = fmaf(v.z, ri, fmaf(v.w, rr, sm.dpi));
    };
    float x, y, z;
    frame_offset(fr, pt, x, y, z);
    const float r2 = x * x + y * y + z * z;
    // orders m and m + 1 advance together (two independent recurrences in n,
    // each with its own sums) so that a lane has two chains in flight
    Sums sa = {0.f, 0.f, 0.f, 0.f}, sb = sa;
    float mre = 1.f, mim = 0.f;  // R^_m^m
#pragma unroll
    for (int m = 0; m <= p; m += 2) {
        if (m > 0) {
            const float f = c_rec_d[m];
            const float nre = f * (x * mre - y * mim), nim = f * (x * mim + y * mre);
            mre = nre;
            mim = nim;
        }
        const bool two = m + 1 <= p;
        float bre = 0.f, bim = 0.f;  // R^_{m+1}^{m+1}
        if (two) {
            const float f = c_rec_d[m + 1];
            bre = f * (x * mre - y * mim);
            bim = f * (x * mim + y * mre);
        }
        int ta = m * (m + 1) / 2 + m;  // term (m, m)
        term(ta, mre, mim, sa);
        float a2r = 0.f, a2i = 0.f, a1r = mre, a1i = mim;  // chain m
        float b2r = 0.f, b2i = 0.f, b1r = bre, b1i = bim;  // chain m + 1
#pragma unroll 2
        for (int n = m + 1; n <= p; ++n) {
            ta += n;  // term (n, m)
            const float aa = c_rec_a[ta] * z, ab = c_rec_b[ta] * r2;
            const float rr = aa * a1r - ab * a2r, ri = aa * a1i - ab * a2i;
            a2r = a1r;
            a2i = a1i;
            a1r = rr;
            a1i = ri;
            term(ta, rr, ri, sa);
            float qr = b1r, qi = b1i;  // n == m + 1: the diagonal itself
            if (n > m + 1) {
                const int tb = ta + 1;
                const float ba = c_rec_a[tb] * z, bb = c_rec_b[tb] * r2;
                qr = ba * b1r - bb * b2r;
                qi = ba * b1i - bb * b2i;
                b2r = b1r;
                b2i = b1i;
                b1r = qr;
                b1i = qi;
            }
            term(ta + 1, qr, qi, sb);
        }
        mre = bre;  // the next pair starts from R^_{m+1}^{m+1}
        mim = bim;
    }
    const float phi = sa.phi + sb.phi, dz = sa.dz + sb.dz, dpr = sa.dpr + sb.dpr, dpi = sa.dpi + sb.dpi;
    return make_float4(phi * inv_s, dpr * inv_s2, dpi * inv_s2, dz * inv_s2);
}

// Particle-parallel L2P.  Warp w takes the sorted particles 32 w .. 32 w + 31,
// whatever leaves they belong to (pcell: the leaf of each sorted particle), so
// every lane has a particle; a leaf of n particles no longer leaves 32 - n
// lanes, or 64 - n in a second pass, without work.  The lanes' leaves form
// runs; the warp builds the records of up to kL2PSlots runs at a time in its own
// shared memory, and each lane evaluates its particle from its run's records.
constexpr int kL2PWarps = 4;  // warps per block
constexpr int kL2PSlots = 3;  // leaves whose records a warp holds at once

template <int PT>
__global__ void __launch_bounds__(32 * kL2PWarps, 6)
    k_l2p(CellArrays c, const int *__restrict__ pcell, int64_t n, const float4 *__restrict__ pts, int p_run,
          int P2pad, const float *__restrict__ L, float4 *__restrict__ far)
{
    const int p = PT > 0 ? PT : p_run;  // compile-time order when PT > 0 (as in k_p2m)
    extern __shared__ float4 l2p_sm[];  // per warp and slot: 2 x ntri records, then P2pad floats of L
    const int ntri = (p + 1) * (p + 2) / 2;
    const int slot_f4 = 2 * ntri + P2pad / 4;  // float4 per slot
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *wsm = l2p_sm + (size_t)warp * kL2PSlots * slot_f4;
    const int64_t i = ((int64_t)blockIdx.x * kL2PWarps + warp) * 32 + lane;
    const bool valid = i < n;
    const int cell = valid ? pcell[i] : -1;
    const int prev = __shfl_up_sync(0xffffffffu, cell, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, valid && (lane == 0 || prev != cell));
    if (heads == 0) return;  // the whole warp is past the particles
    const int nrun = __popc(heads);
    const int myrun = __popc(heads & (0xffffffffu >> (31 - lane))) - 1;  // runs starting at or before this lane
    float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
    Frame fr = {pt, pt};
    if (valid) {
        pt = pts[i];
        fr = cell_frame(c, cell);
    }
    for (int r0 = 0; r0 < nrun; r0 += kL2PSlots) {
#pragma unroll
        for (int s = 0; s < kL2PSlots; ++s) {
            if (r0 + s >= nrun) break;
            // the lane that heads run r0 + s
            const int hl = __ffs(__ballot_sync(0xffffffffu, ((heads >> lane) & 1u) && myrun == r0 + s)) - 1;
            const int rc = __shfl_sync(0xffffffffu, cell, hl);
            float4 *rec = wsm + (size_t)s * slot_f4;
            l2p_records(L + (int64_t)rc * P2pad, p, reinterpret_cast<float *>(rec + 2 * ntri), rec, lane);
        }
        if (valid && myrun >= r0 && myrun < r0 + kL2PSlots)
            far[i] = l2p_eval<PT>(wsm + (size_t)(myrun - r0) * slot_f4, fr, pt, p);
        __syncwarp();
    }
}

size_t l2p_block_smem(int p, int P2pad) { return (size_t)kL2PWarps * kL2PSlots * l2p_smem(p, P2pad); }

void launch_l2p(const CellArrays &c, const int *pcell, int64_t n, const float4 *pts, int p, int P2pad,
                const float *L, float4 *far, cudaStream_t st)
{
    if (n <= 0) return;
    const size_t sh = l2p_block_smem(p, P2pad);
    const unsigned grid = (unsigned)ceil_div(n, (int64_t)32 * kL2PWarps);
    switch (p) {
#define FMM_L2P_CASE(P)                                                          \
    case P:                                                                      \
        set_smem_limit_once((const void *)k_l2p<P>, (int)sh);                     \
        k_l2p<P><<<grid, 32 * kL2PWarps, sh, st>>>(c, pcell, n, pts, p, P2pad, L, far); \
        break;
        FMM_L2P_CASE(4)
        FMM_L2P_CASE(6)
        FMM_L2P_CASE(8)
        FMM_L2P_CASE(10)
        FMM_L2P_CASE(12)
#undef FMM_L2P_CASE
    default:
        set_smem_limit_once((const void *)k_l2p<0>, (int)sh);
        k_l2p<0><<<grid, 32 * kL2PWarps, sh, st>>>(c, pcell, n, pts, p, P2pad, L, far);
    }
    FMM_LAUNCH_CHECK();
}

// Cell-particle (M2P, the treecode kernel): one warp per target leaf with an
// M2P list; every listed source cell's multipole is evaluated at the leaf's
// particles and added to the far field.  With u = (x - c_S) / s_S and the
// order-normalised irregular harmonics I^_n^m = I_n^m / nu_n^m,
//   phi    = (1/s)   sum M^_n^m I^_n^m(u)
//   d/dz   = -(1/s^2) sum M^_n^m I^_{n+1}^m   sqrt((n+1-m)(n+1+m))
//   D+     = (1/s^2) sum [M^_n^m I^_{n+1}^{m+1} sqrt((n+m+1)(n+m+2))
//                          - conj(M^_n^m I^_{n+1}^{m-1}) sqrt((n-m+1)(n-m+2)) (m >= 1)]
// (sums over m >= 0 with weight 2 on the real parts of m > 0 where the signed-m
// sum pairs conjugates), from d/dz I_n^m = -I_{n+1}^m and (d/dx + i d/dy)
// I_n^m = I_{n+1}^{m+1}.  Recurrences of I^: I^_0^0 = 1/r,
// I^_m^m = -sqrt((2m-1)/(2m)) (x + iy)/r^2 I^_{m-1}^{m-1},
// I^_n^m = ((2n-1) z I^_{n-1}^m - sqrt((n+m-1)(n-m-1)) I^_{n-2}^m) / (r^2 sqrt((n+m)(n-m))).
// Particle-cell (P2L): one warp per target cell with a P2L list.  The source
// particles' contributions L^_n^m += q conj(I^_n^m(u)), u = (y - c_T) / s_T
// (the unit-scaled, order-normalised form of L_n^m += q conj(I_n^m(y - c_T))),
// are formed per particle (lane), reduced over the warp through shared memory
// rows as in P2M, and added to the cell's row of L after its M2L sum.
__global__ void __launch_bounds__(32)
    k_p2l(CellArrays c, ListArrays Ls, int ncells, const float4 *__restrict__ pts,
          const double *__restrict__ box, int p, int P2pad, float *__restrict__ L, const int *__restrict__ sz)
{
    extern __shared__ float rows[];  // 32 x (P2pad + 1)
    if (sz) ncells = sz[kSzCells];
    // blocks stride over the cells, so that the grid can be sized to the GPU and a
    // solve without particle-cell pairs costs one pass over the counts
    for (int cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        const int cnt = Ls.p2l_cnt[cell];
        if (cnt == 0) continue;
        const int *slist = Ls.p2l_src + Ls.p2l_off[cell];
        const int lane = threadIdx.x;
        const int stride = P2pad + 1;
        const Frame fr = cell_frame(c, cell);
        float acc[kMaxChunks];
#pragma unroll
        for (int j = 0; j < kMaxChunks; ++j) acc[j] = 0.f;
        float *row = rows + lane * stride;
        for (int k = 0; k < cnt; ++k) {
            const int S = slist[k];
            const int b = c.begin[S], e = c.end[S];
            for (int base = b; base < e; base += 32) {
                const int i = base + lane;
                for (int j = 0; j < P2pad; ++j) row[j] = 0.f;
                if (i < e) {
                    const float4 pt = pts[i];
                    float x, y, z;
                    frame_offset(fr, pt, x, y, z);
                    const float q = pt.w;
                    const float r2 = x * x + y * y + z * z, ir2 = 1.f / r2;
                    float mre = rsqrtf(r2), mim = 0.f;  // I^_m^m
                    for (int m = 0; m <= p; ++m) {
                        if (m > 0) {
                            const float f = c_rec_d[m] * ir2;
                            const float nre = f * (x * mre - y * mim), nim = f * (x * mim + y * mre);
                            mre = nre;
                            mim = nim;
                        }
                        float p2r = 0.f, p2i = 0.f, p1r = mre, p1i = mim;
                        for (int n = m; n <= p; ++n) {
                            float ir, ii;
                            if (n == m) {
                                ir = mre;
                                ii = mim;
                            } else {
                                const int t = n * (n + 1) / 2 + m;
                                const float a = c_rec_a[t] * z * ir2, bb = c_rec_b[t] * ir2;
                                ir = a * p1r - bb * p2r;
                                ii = a * p1i - bb * p2i;
                                p2r = p1r;
                                p2i = p1i;
                                p1r = ir;
                                p1i = ii;
                            }
                            if (m == 0) {
                                row[n * n] = q * ir;
                            } else {
                                row[n * n + 2 * m - 1] = q * ir;
                                row[n * n + 2 * m] = -q * ii;
                            }
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int j = 0; j < kMaxChunks; ++j) {
                    const int kk = lane + 32 * j;
                    if (kk < P2pad) {
                        float sum = 0.f;
                        for (int r = 0; r < 32; ++r) sum += rows[r * stride + kk];
                        acc[j] += sum;
                    }
                }
                __syncwarp();
            }
        }
        const int P2 = nterms(p);
#pragma unroll
        for (int j = 0; j < kMaxChunks; ++j) {
            const int kk = lane + 32 * j;
            if (kk < P2) L[(int64_t)cell * P2pad + kk] += acc[j];
        }
        __syncwarp();  // the warp's shared rows are rewritten for the next cell
    }
}

size_t m2p_smem(int p, int P2pad)
{
    const int nt = (p + 2) * (p + 3) / 2;
    return sizeof(float) * (2 * (size_t)nt + (p + 2) + 3 * (size_t)P2pad + 4 * kM2PWarps +
                            (size_t)kM2PWarps * 4 * P2pad);
}

__global__ void __launch_bounds__(32 * kM2PWarps)
    k_m2p(CellArrays c, ListArrays Ls, const int *__restrict__ leaves, int nleaves,
          const float4 *__restrict__ pts, const double *__restrict__ box, int p, int P2pad,
          const float *__restrict__ M, float4 *__restrict__ far, const int *__restrict__ sz)
{
    extern __shared__ float sm[];
    if (sz) nleaves = sz[kSzLeaves];
    // per block: recurrence coefficients of I^ for (n, m) at n(n+1)/2 + m, n <= p + 1,
    // the diagonal factors, and the three derivative weights per stored coefficient
    const int ntri = (p + 2) * (p + 3) / 2;
    float *ca = sm, *cb = ca + ntri, *cd = cb + ntri, *fz = cd + (p + 2), *f1 = fz + P2pad,
          *f2 = f1 + P2pad, *sgeo = f2 + P2pad, *wbuf = sgeo + 4 * kM2PWarps;
    for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= t) ++n;
        const int m = t - n * (n + 1) / 2;
        const float den = n > m ? rsqrtf((float)((n + m) * (n - m))) : 0.f;
        ca[t] = (2.f * n - 1.f) * den;
        cb[t] = n > m + 1 ? sqrtf((float)((n + m - 1) * (n - m - 1))) * den : 0.f;
    }
    for (int m = threadIdx.x; m <= p + 1; m += blockDim.x) cd[m] = m > 0 ? -sqrtf((2.f * m - 1.f) / (2.f * m)) : 1.f;
    for (int j = threadIdx.x; j < P2pad; j += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 1) <= j) ++n;
        const int m = (j - n * n + 1) / 2;
        fz[j] = sqrtf((float)((n + 1 - m) * (n + 1 + m)));
        f1[j] = sqrtf((float)((n + m + 1) * (n + m + 2)));
        f2[j] = sqrtf((float)((n - m + 1) * (n - m + 2)));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warps stride over the leaves, so that the grid can be sized to the GPU and a
    // solve without cell-particle pairs costs one pass over the counts
    for (int li = blockIdx.x * kM2PWarps + warp; li < nleaves; li += gridDim.x * kM2PWarps) {
        const int cell = leaves[li];
        const int cnt = Ls.m2p_cnt[cell];
        if (cnt == 0) continue;
        const int *slist = Ls.m2p_src + Ls.m2p_off[cell];
        float *Mh = wbuf + warp * 4 * P2pad, *Mz = Mh + P2pad, *Mx1 = Mz + P2pad, *Mx2 = Mx1 + P2pad;
        const int P2 = nterms(p);
        const int b = c.begin[cell], e = c.end[cell];
        // particle offsets from the target leaf's centre in FP32; the shift and scale of
        // each source come from one FP64 evaluation per (leaf, source) pair, not per particle
        double cT[3], sT;
        cell_centre_side(c, cell, box, cT, sT);
        float *geo = sgeo + warp * 4;  // (c_T - c_S) / s_S and s_T / s_S of the current source
        for (int i0 = b; i0 < e; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < e;
            const float4 pt = pts[valid ? i : b];
            const double isT = 1.0 / sT;
            const float rx = (float)(((double)pt.x - cT[0]) * isT), ry = (float)(((double)pt.y - cT[1]) * isT),
                        rz = (float)(((double)pt.z - cT[2]) * isT);
            float phi = 0.f, dz = 0.f, dpr = 0.f, dpi = 0.f;
            for (int k = 0; k < cnt; ++k) {
                const int S = slist[k];
                __syncwarp();
                if (lane == 0) {
                    double cS[3], sS;
                    cell_centre_side(c, S, box, cS, sS);
                    const double isS = 1.0 / sS;  // sides are powers of two times the box side
                    geo[0] = (float)((cT[0] - cS[0]) * isS);
                    geo[1] = (float)((cT[1] - cS[1]) * isS);
                    geo[2] = (float)((cT[2] - cS[2]) * isS);
                    geo[3] = (float)(sT * isS);
                }
                for (int j = lane; j < P2pad; j += 32) {
                    const float v = j < P2 ? M[(int64_t)S * P2pad + j] : 0.f;
                    Mh[j] = v;
                    Mz[j] = v * fz[j];
                    Mx1[j] = v * f1[j];
                    Mx2[j] = v * f2[j];
                }
                __syncwarp();
                const float ratio = geo[3];
                const float x = fmaf(rx, ratio, geo[0]), y = fmaf(ry, ratio, geo[1]), z = fmaf(rz, ratio, geo[2]);
                const float is1 = ratio / (float)sT, is2 = is1 * is1;  // 1 / s_S = (s_T / s_S) / s_T
                const float r2 = x * x + y * y + z * z;
                const float ir2 = 1.f / r2;
                float sphi = 0.f, sdz = 0.f, sdr = 0.f, sdi = 0.f;
                float mre = rsqrtf(r2), mim = 0.f;  // I^_m^m
                for (int m = 0; m <= p + 1; ++m) {
                    if (m > 0) {
                        const float f = cd[m] * ir2;
                        const float nre = f * (x * mre - y * mim), nim = f * (x * mim + y * mre);
                        mre = nre;
                        mim = nim;
                    }
                    const float w = m == 0 ? 1.f : 2.f;
                    float p2r = 0.f, p2i = 0.f, p1r = mre, p1i = mim;
                    for (int n = m; n <= p + 1; ++n) {
                        float ir, ii;
                        if (n == m) {
                            ir = mre;
                            ii = mim;
                        } else {
                            const int t = n * (n + 1) / 2 + m;
                            const float a = ca[t] * z * ir2, bb = cb[t] * ir2;
                            ir = a * p1r - bb * p2r;
                            ii = a * p1i - bb * p2i;
                            p2r = p1r;
                            p2i = p1i;
                            p1r = ir;
                            p1i = ii;
                        }
                        if (n <= p) {  // phi += w Re(M^_n^m I^_n^m)
                            const int k = n * n + (m == 0 ? 0 : 2 * m - 1);
                            const float mr = Mh[k], mi = m == 0 ? 0.f : Mh[k + 1];
                            sphi += w * (mr * ir - mi * ii);
                        }
                        if (n >= 1) {
                            const int n1 = n - 1, base = n1 * n1;
                            if (m <= n1) {  // dz += w Re(Mz_{n-1}^m I^_n^m)
                                const int k = base + (m == 0 ? 0 : 2 * m - 1);
                                const float mr = Mz[k], mi = m == 0 ? 0.f : Mz[k + 1];
                                sdz += w * (mr * ir - mi * ii);
                            }
                            if (m >= 1) {  // D+ += Mx1_{n-1}^{m-1} I^_n^m
                                const int mm = m - 1;
                                const int k = base + (mm == 0 ? 0 : 2 * mm - 1);
                                const float mr = Mx1[k], mi = mm == 0 ? 0.f : Mx1[k + 1];
                                sdr += mr * ir - mi * ii;
                                sdi += mr * ii + mi * ir;
                            }
                            if (m + 1 <= n1) {  // D+ -= conj(Mx2_{n-1}^{m+1} I^_n^m)
                                const int k = base + 2 * (m + 1) - 1;
                                const float mr = Mx2[k], mi = Mx2[k + 1];
                                sdr -= mr * ir - mi * ii;
                                sdi += mr * ii + mi * ir;
                            }
                        }
                    }
                }
                phi += sphi * is1;
                dz -= sdz * is2;
                dpr += sdr * is2;
                dpi += sdi * is2;
            }
            if (valid) {
                float4 f = far[i];
                f.x += phi;
                f.y += dpr;
                f.z += dpi;
                f.w += dz;
                far[i] = f;
            }
        }
        __syncwarp();  // the warp's shared rows are rewritten for the next cell
    }
}

}  // namespace fmm
