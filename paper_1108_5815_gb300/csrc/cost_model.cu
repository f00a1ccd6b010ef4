// cost_model.cu -- kernel pre-calculation and the learned cost model (host side).
//
// Section "Kernel pre-calculation": every interaction kernel is run on
// artificial coordinates and charges and its execution time is measured; the
// traversal then picks the cheapest interaction type.  The paper also notes that
// on a GPU the time does not scale with the problem size, because larger launches
// fill the device better; so the artificial launches here are sized like real
// solves (tens of thousands of target leaves, 27 source cells each), and the
// time per pair is taken from a full launch.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "cost_model.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ uint64_t splitmix(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float unit(uint64_t z) { return (float)(z >> 40) * (1.0f / 16777216.0f); }

__global__ void k_synth_points(float4 *__restrict__ pts, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = seed + 4 * (uint64_t)i;
        pts[i] = make_float4(unit(splitmix(b)), unit(splitmix(b + 1)), unit(splitmix(b + 2)),
                             2.f * unit(splitmix(b + 3)) - 1.f);
    }
}

__global__ void k_synth_uniform(float *__restrict__ xyz, float *__restrict__ q, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = seed + 4 * (uint64_t)i;
        xyz[3 * i] = unit(splitmix(b));
        xyz[3 * i + 1] = unit(splitmix(b + 1));
        xyz[3 * i + 2] = unit(splitmix(b + 2));
        q[i] = 2.f * unit(splitmix(b + 3)) - 1.f;
    }
}

// Points of a Plummer sphere of scale 1, cut at radius 20 through the mass
// fraction (M(r) = r^3 / (1 + r^2)^(3/2), M(20) = 0.9963): r from the fraction m
// as 1 / sqrt(m^(-2/3) - 1), the direction uniform on the sphere; charges 1/n.
__global__ void k_synth_plummer(float *__restrict__ xyz, float *__restrict__ q, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = seed + 4 * (uint64_t)i;
        const float m = fmaxf(0.9963f * unit(splitmix(b)), 1e-6f);
        const float r = rsqrtf(powf(m, -2.f / 3.f) - 1.f);
        const float z = 2.f * unit(splitmix(b + 1)) - 1.f;
        const float ph = 6.2831853f * unit(splitmix(b + 2));
        const float sxy = sqrtf(fmaxf(0.f, 1.f - z * z));
        float sp, cp;
        sincosf(ph, &sp, &cp);
        xyz[3 * i] = r * sxy * cp;
        xyz[3 * i + 1] = r * sxy * sp;
        xyz[3 * i + 2] = r * z;
        q[i] = 1.f / (float)n;
    }
}

// nL target leaves of nt particles, nS source cells of ns particles; leaf t
// lists K sources spread over the source cells.
__global__ void k_synth_lists(int nL, int nt, int nS, int ns, int K, int *__restrict__ begin,
                              int *__restrict__ end, int *__restrict__ off, int *__restrict__ cnt,
                              int *__restrict__ src, int *__restrict__ leaves)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nL) {
        begin[i] = i * nt;
        end[i] = (i + 1) * nt;
        off[i] = i * K;
        cnt[i] = K;
        leaves[i] = i;
        for (int k = 0; k < K; ++k) src[(int64_t)i * K + k] = nL + (int)(((int64_t)i * 131 + k * 7) % nS);
    }
    if (i < nS) {
        begin[nL + i] = nL * nt + i * ns;
        end[nL + i] = nL * nt + (i + 1) * ns;
    }
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    explicit DevBuf(size_t n) { FMM_CUDA_TRY(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T))); }
    ~DevBuf() { cudaFree(p); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

double interp_axis(const std::vector<double> &xs, double x, size_t &i0)
{
    // segment index and weight of x on the grid xs (linear extrapolation beyond the ends)
    const size_t n = xs.size();
    size_t i = 0;
    while (i + 2 < n && x > xs[i + 1]) ++i;
    i0 = i;
    return (x - xs[i]) / (xs[i + 1] - xs[i]);
}

}  // namespace

std::vector<P2PTiming> pretime_p2p(const std::vector<int> &counts, uint64_t seed, cudaStream_t st)
{
    constexpr int K = 27;
    constexpr int64_t kMaxTargets = 1 << 24, kMaxSources = 1 << 22, kMaxLeaves = 1 << 16;
    const int cmax = *std::max_element(counts.begin(), counts.end());
    DevBuf<float4> pts(kMaxTargets + kMaxSources), near(kMaxTargets);
    DevBuf<int> begin(2 * kMaxLeaves), end(2 * kMaxLeaves), off(kMaxLeaves), cnt(kMaxLeaves),
        src(kMaxLeaves * K), leaves(kMaxLeaves);
    k_synth_points<<<1024, 256, 0, st>>>(pts.p, kMaxTargets + kMaxSources, seed);
    FMM_LAUNCH_CHECK();
    (void)cmax;
    int nsm = 152, dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    set_carveout_once((const void *)k_p2p, cudaSharedmemCarveoutMaxShared);
    cudaEvent_t e0, e1;
    FMM_CUDA_TRY(cudaEventCreate(&e0));
    FMM_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<P2PTiming> out;
    for (int nt : counts) {
        for (int ns : counts) {
            const double inter = (double)K * nt * ns;
            int64_t nL = (int64_t)std::llround((double)(1 << 27) / inter);
            nL = std::max<int64_t>(nL, (int64_t)nsm * 8);  // at least 8 leaves per SM
            nL = std::min<int64_t>({nL, kMaxLeaves, kMaxTargets / nt});
            const int64_t nS = std::min<int64_t>(std::max<int64_t>(nL, K), std::min<int64_t>(kMaxLeaves, kMaxSources / ns));
            CellArrays c{};
            c.begin = begin.p;
            c.end = end.p;
            ListArrays L{};
            L.p2p_off = off.p;
            L.p2p_cnt = cnt.p;
            L.p2p_src = src.p;
            const int64_t nmax = std::max(nL, nS);
            k_synth_lists<<<(unsigned)ceil_div(nmax, 256), 256, 0, st>>>((int)nL, nt, (int)nS, ns, K, begin.p,
                                                                         end.p, off.p, cnt.p, src.p, leaves.p);
            FMM_LAUNCH_CHECK();
            float best = 1e30f;
            for (int rep = 0; rep < 4; ++rep) {
                FMM_CUDA_TRY(cudaEventRecord(e0, st));
                k_p2p<<<(unsigned)std::max<int64_t>(1, nL), 32, 0, st>>>(c, L, leaves.p, (int)nL, pts.p, near.p);
                FMM_LAUNCH_CHECK();
                FMM_CUDA_TRY(cudaEventRecord(e1, st));
                FMM_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                FMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0) best = std::min(best, ms);  // the first run warms up
            }
            out.push_back({nt, ns, (double)best * 1e6 / ((double)nL * K)});
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

std::vector<double> pretime_m2p(int p, const std::vector<int> &counts, uint64_t seed, cudaStream_t st)
{
    constexpr int K = 27, kLevel = 6;
    constexpr int64_t kMaxTargets = 1 << 22, kMaxLeaves = 1 << 14;
    const int P2pad = nterms_pad(p);
    DevBuf<float4> pts(kMaxTargets), far(kMaxTargets);
    DevBuf<int> begin(2 * kMaxLeaves), end(2 * kMaxLeaves), off(kMaxLeaves), cnt(kMaxLeaves),
        src(kMaxLeaves * K), leaves(kMaxLeaves), level(2 * kMaxLeaves), sys(2 * kMaxLeaves);
    DevBuf<uint64_t> prefix(2 * kMaxLeaves);
    DevBuf<float> M((size_t)2 * kMaxLeaves * P2pad);  // rows of every cell id (targets and sources)
    DevBuf<double> box(4);
    k_synth_points<<<1024, 256, 0, st>>>(pts.p, kMaxTargets, seed);
    FMM_LAUNCH_CHECK();
    // multipole rows: small artificial values (the kernel's cost does not depend on them)
    k_synth_points<<<1024, 256, 0, st>>>(reinterpret_cast<float4 *>(M.p), (int64_t)2 * kMaxLeaves * P2pad / 4,
                                         seed + 1);
    FMM_LAUNCH_CHECK();
    const double hbox[4] = {0.0, 0.0, 0.0, 1.0};
    FMM_CUDA_TRY(cudaMemcpyAsync(box.p, hbox, sizeof(hbox), cudaMemcpyHostToDevice, st));
    std::vector<int> hl(2 * kMaxLeaves, kLevel), hs(2 * kMaxLeaves, 0);
    std::vector<uint64_t> hp(2 * kMaxLeaves);
    for (int64_t i = 0; i < 2 * kMaxLeaves; ++i) hp[i] = (uint64_t)((i * 2654435761ull) & ((1ull << (3 * kLevel)) - 1));
    FMM_CUDA_TRY(cudaMemcpyAsync(level.p, hl.data(), sizeof(int) * hl.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(sys.p, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(prefix.p, hp.data(), sizeof(uint64_t) * hp.size(), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    FMM_CUDA_TRY(cudaEventCreate(&e0));
    FMM_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<double> out;
    for (int nt : counts) {
        int64_t nL = std::min<int64_t>(kMaxLeaves, kMaxTargets / nt);
        const int64_t nS = kMaxLeaves;
        CellArrays c{};
        c.begin = begin.p;
        c.end = end.p;
        c.level = level.p;
        c.prefix = prefix.p;
        c.sys = sys.p;
        ListArrays L{};
        L.m2p_off = off.p;
        L.m2p_cnt = cnt.p;
        L.m2p_src = src.p;
        // sources get one particle each; only their multipoles are read
        k_synth_lists<<<(unsigned)ceil_div(nS, 256), 256, 0, st>>>((int)nL, nt, (int)nS, 1, K, begin.p, end.p,
                                                                   off.p, cnt.p, src.p, leaves.p);
        FMM_LAUNCH_CHECK();
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            FMM_CUDA_TRY(cudaEventRecord(e0, st));
            const size_t sh = m2p_smem(p, P2pad);
            if (sh > 48 * 1024) set_smem_limit_once((const void *)k_m2p, (int)sh);
            k_m2p<<<(unsigned)ceil_div(nL, kM2PWarps), 32 * kM2PWarps, sh, st>>>(c, L, leaves.p, (int)nL, pts.p,
                                                                                 box.p, p, P2pad, M.p, far.p);
            FMM_LAUNCH_CHECK();
            FMM_CUDA_TRY(cudaEventRecord(e1, st));
            FMM_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            FMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = std::min(best, ms);
        }
        out.push_back((double)best * 1e6 / ((double)nL * K));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

std::vector<double> pretime_p2l(int p, const std::vector<int> &counts, uint64_t seed, cudaStream_t st)
{
    constexpr int K = 27, kLevel = 6;
    constexpr int64_t kMaxSources = 1 << 22, kMaxCells = 1 << 14;
    const int P2pad = nterms_pad(p);
    DevBuf<float4> pts(kMaxSources);
    DevBuf<int> begin(2 * kMaxCells), end(2 * kMaxCells), off(kMaxCells), cnt(kMaxCells), src(kMaxCells * K),
        leaves(kMaxCells), level(2 * kMaxCells), sys(2 * kMaxCells);
    DevBuf<uint64_t> prefix(2 * kMaxCells);
    DevBuf<float> L((size_t)2 * kMaxCells * P2pad);
    DevBuf<double> box(4);
    DevBuf<int4> geom(2 * kMaxCells);
    DevBuf<float4> fhi(2 * kMaxCells), flo(2 * kMaxCells);
    k_synth_points<<<1024, 256, 0, st>>>(pts.p, kMaxSources, seed);
    FMM_LAUNCH_CHECK();
    const double hbox[4] = {0.0, 0.0, 0.0, 1.0};
    FMM_CUDA_TRY(cudaMemcpyAsync(box.p, hbox, sizeof(hbox), cudaMemcpyHostToDevice, st));
    std::vector<int> hl(2 * kMaxCells, kLevel), hs(2 * kMaxCells, 0);
    std::vector<uint64_t> hp(2 * kMaxCells);
    for (int64_t i = 0; i < 2 * kMaxCells; ++i) hp[i] = (uint64_t)((i * 2654435761ull) & ((1ull << (3 * kLevel)) - 1));
    FMM_CUDA_TRY(cudaMemcpyAsync(level.p, hl.data(), sizeof(int) * hl.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(sys.p, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(prefix.p, hp.data(), sizeof(uint64_t) * hp.size(), cudaMemcpyHostToDevice, st));
    {
        // the cells' FP32 frames (the particle offsets of k_p2l)
        CellArrays g{};
        g.level = level.p;
        g.prefix = prefix.p;
        g.sys = sys.p;
        g.geom = geom.p;
        g.fhi = fhi.p;
        g.flo = flo.p;
        k_cell_geom<<<(unsigned)ceil_div(2 * kMaxCells, 256), 256, 0, st>>>(g, (int)(2 * kMaxCells), box.p);
        FMM_LAUNCH_CHECK();
    }
    const size_t sh = (size_t)32 * (P2pad + 1) * sizeof(float);
    if (sh > 48 * 1024) set_smem_limit_once((const void *)k_p2l, (int)sh);
    cudaEvent_t e0, e1;
    FMM_CUDA_TRY(cudaEventCreate(&e0));
    FMM_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<double> out;
    for (int ns : counts) {
        const int64_t nS = std::min<int64_t>(kMaxCells, kMaxSources / ns);
        const int64_t nT = std::min<int64_t>(kMaxCells, std::max<int64_t>(1216, (int64_t)(1 << 24) / ((int64_t)K * ns)));
        CellArrays c{};
        c.begin = begin.p;
        c.end = end.p;
        c.level = level.p;
        c.prefix = prefix.p;
        c.sys = sys.p;
        c.geom = geom.p;
        c.fhi = fhi.p;
        c.flo = flo.p;
        ListArrays Ls{};
        Ls.p2l_off = off.p;
        Ls.p2l_cnt = cnt.p;
        Ls.p2l_src = src.p;
        // targets hold no particles of their own; sources get ns particles each
        k_synth_lists<<<(unsigned)ceil_div(std::max(nS, nT), 256), 256, 0, st>>>((int)nT, 0, (int)nS, ns, K, begin.p,
                                                                                  end.p, off.p, cnt.p, src.p, leaves.p);
        FMM_LAUNCH_CHECK();
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            FMM_CUDA_TRY(cudaEventRecord(e0, st));
            k_p2l<<<(unsigned)nT, 32, sh, st>>>(c, Ls, (int)nT, pts.p, box.p, p, P2pad, L.p);
            FMM_LAUNCH_CHECK();
            FMM_CUDA_TRY(cudaEventRecord(e1, st));
            FMM_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            FMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = std::min(best, ms);
        }
        out.push_back((double)best * 1e6 / ((double)nT * K));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

void table_from_timings(const std::vector<P2PTiming> &grid, double m2l_ns, const std::vector<int> &m2p_counts,
                        const std::vector<double> &m2p_ns, const std::vector<double> &p2l_ns, uint8_t *sel)
{
    // ln(time per pair) on the (log2 nt, log2 ns) grid, bilinear in the logs
    std::vector<int> cs;
    for (const auto &g : grid) cs.push_back(g.nt);
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    const size_t n = cs.size();
    std::vector<double> lx(n);
    for (size_t i = 0; i < n; ++i) lx[i] = std::log2((double)cs[i]);
    std::vector<double> lt(n * n, 0.0);
    for (const auto &g : grid) {
        const size_t i = std::lower_bound(cs.begin(), cs.end(), g.nt) - cs.begin();
        const size_t j = std::lower_bound(cs.begin(), cs.end(), g.ns) - cs.begin();
        lt[i * n + j] = std::log(g.ns_per_pair);
    }
    const double lm = std::log(m2l_ns);
    std::vector<double> qx, qt, lt_p2l;
    for (size_t i = 0; i < m2p_ns.size(); ++i) {
        qx.push_back(std::log2((double)m2p_counts[i]));
        qt.push_back(std::log(m2p_ns[i]));
    }
    for (size_t i = 0; i < p2l_ns.size(); ++i) lt_p2l.push_back(std::log(p2l_ns[i]));
    for (int bt = 0; bt < kSelNB; ++bt) {
        size_t i0;
        const double wi = interp_axis(lx, bucket_mid_log2(bt), i0);
        double lq = 1e300;  // ln of the M2P time per pair at this target count
        if (qx.size() >= 2) {
            size_t q0;
            const double wq = interp_axis(qx, bucket_mid_log2(bt), q0);
            lq = (1 - wq) * qt[q0] + wq * qt[q0 + 1];
        }
        for (int bs = 0; bs < kSelNB; ++bs) {
            size_t j0;
            const double wj = interp_axis(lx, bucket_mid_log2(bs), j0);
            const double a = lt[i0 * n + j0], b = lt[i0 * n + j0 + 1], c = lt[(i0 + 1) * n + j0],
                         d = lt[(i0 + 1) * n + j0 + 1];
            const double v = (1 - wi) * ((1 - wj) * a + wj * b) + wi * ((1 - wj) * c + wj * d);
            double lp2l = 1e300;  // ln of the P2L time per pair at this source count
            if (lt_p2l.size() >= 2 && lt_p2l.size() == qx.size()) {
                size_t s0;
                const double ws = interp_axis(qx, bucket_mid_log2(bs), s0);
                lp2l = (1 - ws) * lt_p2l[s0] + ws * lt_p2l[s0 + 1];
            }
            uint8_t kind = v < lm ? 1 : 0;
            double best = std::min(v, lm);
            if (lq < best) {
                kind = 2;
                best = lq;
            }
            if (lp2l < best) kind = 3;
            sel[bt * kSelNB + bs] = kind;
        }
    }
}

void synth_plummer(float *xyz, float *q, int64_t n, uint64_t seed, cudaStream_t st)
{
    k_synth_plummer<<<1024, 256, 0, st>>>(xyz, q, n, seed);
    FMM_LAUNCH_CHECK();
}

void synth_uniform(float *xyz, float *q, int64_t n, uint64_t seed, cudaStream_t st)
{
    k_synth_uniform<<<1024, 256, 0, st>>>(xyz, q, n, seed);
    FMM_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ the network

CostModel::~CostModel()
{
    for (void *p : {(void *)w16, (void *)w32, (void *)mom, (void *)vel, (void *)grad, (void *)loss,
                    (void *)inv_cnt, (void *)step, (void *)x, (void *)t, (void *)m, (void *)partial,
                    (void *)loss_part})
        if (p) cudaFree(p);
}

void CostModel::ensure(int64_t n)
{
    if (!w16) {
        FMM_CUDA_TRY(cudaMalloc(&w16, sizeof(__half) * kMlpParams));
        FMM_CUDA_TRY(cudaMalloc(&w32, sizeof(float) * kMlpParams));
        FMM_CUDA_TRY(cudaMalloc(&mom, sizeof(float) * kMlpParams));
        FMM_CUDA_TRY(cudaMalloc(&vel, sizeof(float) * kMlpParams));
        FMM_CUDA_TRY(cudaMalloc(&grad, sizeof(float) * kMlpParams));
        FMM_CUDA_TRY(cudaMalloc(&loss, sizeof(float)));
        FMM_CUDA_TRY(cudaMalloc(&inv_cnt, sizeof(float)));
        FMM_CUDA_TRY(cudaMalloc(&step, sizeof(int)));
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)mlp_grad_smem()));
    }
    if (n > cap) {
        for (float **p : {&x, &t, &m, &partial, &loss_part})
            if (*p) {
                cudaFree(*p);
                *p = nullptr;
            }
        const int64_t nb = ceil_div(n, 64);
        FMM_CUDA_TRY(cudaMalloc(&x, sizeof(float) * 4 * n));
        FMM_CUDA_TRY(cudaMalloc(&t, sizeof(float) * 2 * n));
        FMM_CUDA_TRY(cudaMalloc(&m, sizeof(float) * 2 * n));
        FMM_CUDA_TRY(cudaMalloc(&partial, sizeof(float) * kMlpParams * nb));
        FMM_CUDA_TRY(cudaMalloc(&loss_part, sizeof(float) * nb));
        cap = n;
    }
}

void model_set(CostModel &cm, const float *params, cudaStream_t st)
{
    cm.ensure(1);
    std::vector<__half> h(kMlpParams);
    for (int i = 0; i < kMlpParams; ++i) h[i] = __float2half_rn(params[i]);
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.w32, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.w16, h.data(), sizeof(__half) * kMlpParams, cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemsetAsync(cm.mom, 0, sizeof(float) * kMlpParams, st));
    FMM_CUDA_TRY(cudaMemsetAsync(cm.vel, 0, sizeof(float) * kMlpParams, st));
    FMM_CUDA_TRY(cudaMemsetAsync(cm.step, 0, sizeof(int), st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

std::vector<float> model_init(const Samples &s, uint64_t seed)
{
    SplitMix64 rng{seed};
    std::vector<float> w(kMlpParams, 0.f);
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) w[off + i] = (float)((2.0 * rng.uniform() - 1.0) * a);
    };
    fill(kOffW1, kMlpHidden, kMlpIn);
    fill(kOffW2, kMlpHidden, kMlpHidden);
    fill(kOffW3, kMlpOut, kMlpHidden);
    for (int k = 0; k < kMlpOut; ++k) {
        double sum = 0, cnt = 0;
        for (int64_t i = 0; i < s.size(); ++i) {
            sum += s.m[2 * i + k] * s.t[2 * i + k];
            cnt += s.m[2 * i + k];
        }
        w[kOffB3 + k] = cnt > 0 ? (float)(sum / cnt) : 0.f;
    }
    return w;
}

namespace {

void upload_batch(CostModel &cm, const Samples &s, cudaStream_t st)
{
    const int64_t n = s.size();
    cm.ensure(n);
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.x, s.x.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.t, s.t.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.m, s.m.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, st));
    k_mlp_mask_count<<<1, 256, 0, st>>>(cm.m, (int)(2 * n), cm.inv_cnt);
    FMM_LAUNCH_CHECK();
}

void launch_grad(CostModel &cm, int64_t n, cudaStream_t st)
{
    const int nb = (int)ceil_div(n, 64);
    k_mlp_grad_partial<<<nb, 64, mlp_grad_smem(), st>>>(cm.w16, cm.x, cm.t, cm.m, (int)n, cm.inv_cnt,
                                                        cm.partial, cm.loss_part);
    FMM_LAUNCH_CHECK();
    k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, st>>>(cm.partial, nb, cm.loss_part, cm.grad, cm.loss);
    FMM_LAUNCH_CHECK();
}

void launch_adam(CostModel &cm, float lr, cudaStream_t st)
{
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(cm.w32, cm.mom, cm.vel, cm.grad, cm.w16, cm.step,
                                                         lr, 0.9f, 0.999f, 1e-8f);
    FMM_LAUNCH_CHECK();
    k_mlp_step_inc<<<1, 1, 0, st>>>(cm.step);
    FMM_LAUNCH_CHECK();
}

}  // namespace

void model_grad(CostModel &cm, const Samples &s, float *loss, float *grad, cudaStream_t st)
{
    upload_batch(cm, s, st);
    launch_grad(cm, s.size(), st);
    FMM_CUDA_TRY(cudaMemcpyAsync(loss, cm.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(grad, cm.grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void model_adam_step(CostModel &cm, const Samples &s, float lr, float *loss, cudaStream_t st)
{
    upload_batch(cm, s, st);
    launch_grad(cm, s.size(), st);
    launch_adam(cm, lr, st);
    FMM_CUDA_TRY(cudaMemcpyAsync(loss, cm.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void model_train(CostModel &cm, const Samples &s, int steps, float lr, float &loss0, float &loss1,
                 cudaStream_t st)
{
    upload_batch(cm, s, st);
    // one training step, captured once and replayed
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FMM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        launch_grad(cm, s.size(), st);
        launch_adam(cm, lr, st);
    } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    FMM_CUDA_TRY(cudaStreamEndCapture(st, &graph));
    FMM_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    loss0 = loss1 = 0.f;
    try {
        for (int i = 0; i < steps; ++i) {
            FMM_CUDA_TRY(cudaGraphLaunch(exec, st));
            if (i == 0) FMM_CUDA_TRY(cudaMemcpyAsync(&loss0, cm.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        }
        launch_grad(cm, s.size(), st);
        FMM_CUDA_TRY(cudaMemcpyAsync(&loss1, cm.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        cudaGraphExecDestroy(exec);
        throw;
    }
    g_launch_count += 4 * (int64_t)steps;  // kernels replayed by the graph
    cudaGraphExecDestroy(exec);
}

void model_predict(CostModel &cm, const float *x, int64_t n, float *y, cudaStream_t st)
{
    cm.ensure(n);
    FMM_CUDA_TRY(cudaMemcpyAsync(cm.x, x, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st));
    k_mlp_forward<<<(unsigned)ceil_div(std::max<int64_t>(n, 1), 128), 128, 0, st>>>(cm.w16, cm.x, (int)n, cm.t);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaMemcpyAsync(y, cm.t, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void model_table(CostModel &cm, int p, double theta, uint8_t *sel, cudaStream_t st)
{
    cm.ensure(kSelNB * kSelNB);
    uint8_t *d = reinterpret_cast<uint8_t *>(cm.m);  // scratch, at least 2 * 16384 floats
    k_mlp_table<<<kSelNB * kSelNB / 128, 128, 0, st>>>(cm.w16, (float)p, (float)(1.0 / theta), d);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaMemcpyAsync(sel, d, kSelNB * kSelNB, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace fmm
