// m2l.cu -- M2L translations as offset-grouped dense products (FP32 CUDA cores).
//
// The paper's cell-cell interaction (M2L, O(p^4), sections "Hybrid
// treecode/FMM algorithm" and Fig. "roofline") is, for one (target, source)
// pair, a real (P2 x P2) matrix T(class) applied to the source multipole.  The
// matrix depends only on the pair's offset class (level difference and
// centre offset in cell units), so the translations are regrouped:
//   * targets form tiles of up to 128 cells (the children with one common
//     octant of up to 128 consecutive split parents), so their interaction
//     stencils coincide;
//   * for each tile, every offset class present among its targets is one
//     "block": a 128 x P2 gather of source multipoles (zero rows where a
//     target has no source of that class) times T(class)^T;
//   * a tile's local expansions accumulate over its blocks in registers and
//     are written once.
// This file holds the FP32 CUDA-core version (register-blocked SGEMM, 8 x TN
// outputs per thread).
#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

constexpr int kKc = 16;  // K chunk

template <int NB>
__global__ void __launch_bounds__(256)
    k_m2l_simt(const int *__restrict__ entry_base, const int *__restrict__ entry_class,
               const int *__restrict__ src, const int *__restrict__ tile_cells,
               const float *__restrict__ M, const float *__restrict__ table, int P2pad,
               float *__restrict__ L)
{
    constexpr int TN = NB / 16;
    __shared__ __align__(16) float As[kKc][kTile + 4];
    __shared__ __align__(16) float Bs[kKc][NB + 4];
    __shared__ int s_src[kTile];
    const int tile = blockIdx.x;
    const int n0 = blockIdx.y * NB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    const int eb = entry_base[tile], ee = entry_base[tile + 1];
    for (int e = eb; e < ee; ++e) {
        __syncthreads();
        if (threadIdx.x < kTile) s_src[threadIdx.x] = src[(int64_t)e * kTile + threadIdx.x];
        __syncthreads();
        const float *T = table + (int64_t)entry_class[e] * P2pad * P2pad;
        for (int k0 = 0; k0 < P2pad; k0 += kKc) {
            for (int r = threadIdx.x; r < kTile * 4; r += 256) {
                const int row = r >> 2, q4 = r & 3;
                const int s = s_src[row];
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (s >= 0) v = *reinterpret_cast<const float4 *>(M + (int64_t)s * P2pad + k0 + q4 * 4);
                As[q4 * 4 + 0][row] = v.x;
                As[q4 * 4 + 1][row] = v.y;
                As[q4 * 4 + 2][row] = v.z;
                As[q4 * 4 + 3][row] = v.w;
            }
            for (int r = threadIdx.x; r < NB * 4; r += 256) {
                const int row = r >> 2, q4 = r & 3;
                const float4 v =
                    *reinterpret_cast<const float4 *>(T + (int64_t)(n0 + row) * P2pad + k0 + q4 * 4);
                Bs[q4 * 4 + 0][row] = v.x;
                Bs[q4 * 4 + 1][row] = v.y;
                Bs[q4 * 4 + 2][row] = v.z;
                Bs[q4 * 4 + 3][row] = v.w;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kKc; ++kk) {
                float a[8], b[TN];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = As[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cell = tile_cells[(int64_t)tile * kTile + ty * 8 + i];
        if (cell < 0) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) L[(int64_t)cell * P2pad + n0 + tx * TN + j] = acc[i][j];
    }
}

}  // namespace

void launch_m2l_simt(int ntiles, const int *entry_base, const int *entry_class, const int *src,
                     const int *tile_cells, const float *M, const float *table, int P2pad,
                     float *L, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (P2pad % 128 == 0) {
        dim3 g(ntiles, P2pad / 128);
        k_m2l_simt<128><<<g, 256, 0, st>>>(entry_base, entry_class, src, tile_cells, M, table,
                                           P2pad, L);
    } else if (P2pad % 96 == 0 && P2pad <= 96) {
        dim3 g(ntiles, 1);
        k_m2l_simt<96><<<g, 256, 0, st>>>(entry_base, entry_class, src, tile_cells, M, table,
                                          P2pad, L);
    } else if (P2pad % 64 == 0) {
        dim3 g(ntiles, P2pad / 64);
        k_m2l_simt<64><<<g, 256, 0, st>>>(entry_base, entry_class, src, tile_cells, M, table,
                                          P2pad, L);
    } else {
        dim3 g(ntiles, P2pad / 32);
        k_m2l_simt<32><<<g, 256, 0, st>>>(entry_base, entry_class, src, tile_cells, M, table,
                                          P2pad, L);
    }
    FMM_LAUNCH_CHECK();
}

}  // namespace fmm
