// fmm_api.cu -- C ABI entry points and the host orchestration of one solve.
//
// One solve, on the caller's stream (declared in include/fmm.h):
//   box -> Morton keys -> radix sort -> permute         (tree build: the paper
//   -> adaptive octree level by level                     runs it on the CPU)
//   -> dual tree traversal level by level -> offset classes and M2L tiles
//   -> P2M, M2M (upward) -> M2L -> L2L, L2P (downward) -> P2P -> combine.
// Sizes that depend on the data (cells per level, list lengths, classes) are
// read back once per level through a pinned buffer; every buffer is sized
// exactly from those counts, so no list can overflow.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "cost_model.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace fmm {

static thread_local std::string g_last_error;
thread_local int64_t g_launch_count = 0;
void set_last_error(const std::string &msg) { g_last_error = msg; }

void set_carveout_once(const void *func, int carveout)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> done;
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find({dev, func});
    if (it != done.end() && it->second == carveout) return;
    FMM_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, carveout));
    done[{dev, func}] = carveout;
}

void set_smem_limit_once(const void *func, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> done;
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    int &cur = done[{dev, func}];
    if (cur >= bytes) return;
    FMM_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    cur = bytes;
}

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Calibration of the N_crit pick (solve_calibration): ns per cell and per M2L
// (tile, class) block, and for each calibration solve its P2P kernel time and its
// P2P pairs binned by count bucket (to scale the network's P2P prediction).
struct SolveCal {
    double ns_cell = 0.0, ns_block = 0.0, ns_fixed = 0.0;  // slopes, and the lines' intercepts
    double p2p_ns[2] = {0.0, 0.0};
    std::vector<unsigned long long> hist[2];
};

struct Workspace {
    int device = 0;
    std::mutex mu;
    std::map<std::string, Buf> bufs;
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    // pinned arena for host -> device uploads of one solve (bump allocated)
    unsigned char *up = nullptr;
    size_t up_bytes = 0, up_off = 0;
    // operator caches
    int cache_p = -1;
    std::unordered_map<uint64_t, int> class_cache;
    int table_slots = 0;
    int split_prec = -1, split_slots = 0;  // hi/lo split class matrices: precision and slots done
    // last solve (for fmm_export)
    bool have_solve = false;
    int64_t N = 0;
    int ncells = 0, nleaves = 0, depth = 0, P2pad = 0, nclass = 0;
    int64_t nm2l = 0, np2p = 0;
    int nsys = 1;
    int64_t cap_m2l = 0, cap_p2p = 0, cap_def = 0, cap_m2p = 0, cap_p2l = 0;  // capacities that sufficed
    int64_t nm2p = 0, np2l = 0;
    std::vector<uint8_t> sel_host;                   // selection table of the last solve
    // sizes of the last solve: a plan takes its capacities from them
    struct Shape {
        std::vector<int> lstart;  // first cell of each level, then the cell count
        int64_t N = 0;
        int nsys = 0, ncrit = 0, max_depth = 0;
        int ncells = 0, nleaves = 0, ntiles = 0, nclass = 0, nent = 0, nunits = 0, chunk = 8;
        int64_t tot[5] = {0, 0, 0, 0, 0};  // M2L, P2P, deferred, M2P, P2L pairs
    } shape;
    // hybrid selection: pre-timed kernels and the learned model
    std::vector<P2PTiming> p2p_grid;                      // P2P time per pair on artificial leaves
    std::map<std::tuple<int, uint64_t, int>, double> m2l_ns;  // (p, theta bits, precision) -> ns per pair
    std::map<std::tuple<int, uint64_t, int>, SolveCal> cell_ns;  // (p, theta bits, precision) -> calibration
    std::map<int, std::vector<double>> m2p_ns;                // p -> ns per pair for kSelCounts
    std::map<int, std::vector<double>> p2l_ns;                // p -> ns per pair for kSelCounts
    std::map<std::tuple<int, uint64_t, int, int>, std::vector<uint8_t>> tables;  // (mode, theta, p, prec)
    CostModel cm;
    // The solve runs on two library streams, both non-blocking (a kernel on the
    // legacy default stream would keep the other stream's work from overlapping):
    // main_stream for the tree, traversal and P2P, far_stream (high priority) for
    // the far-field chain.  They are ordered after the caller's stream on entry
    // and the caller's stream is ordered after them on exit.
    cudaStream_t main_stream = nullptr, far_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_tree = nullptr, ev_fork = nullptr, ev_join = nullptr, ev_out = nullptr,
                ev_read = nullptr;
    // Repeated solves (fmm_options.replay): what a solve depends on besides the
    // particle data, the plan captured when a solve repeated its predecessor's
    // key, and that predecessor's key.
    struct ReplayKey {
        int64_t N = 0;
        int nsys = 0, p = 0, ncrit = 0, max_depth = 0, precision = 0, select_mode = 0, unit_blocks = 0;
        double theta = 0.0;
        std::vector<int64_t> off;  // system offsets (batched)
        std::vector<uint8_t> sel;  // the selection table's content (empty: plain FMM)
        bool operator==(const ReplayKey &k) const
        {
            return N == k.N && nsys == k.nsys && p == k.p && ncrit == k.ncrit && max_depth == k.max_depth &&
                   precision == k.precision && select_mode == k.select_mode && unit_blocks == k.unit_blocks &&
                   theta == k.theta && off == k.off && sel == k.sel;
        }
    };
    fmm_plan *replay_plan = nullptr;
    ReplayKey replay_key, last_key;
    bool have_last = false;
};

std::mutex g_ws_mu;
std::map<int, std::unique_ptr<Workspace>> g_ws;

Workspace &workspace_for_current_device()
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto &w = g_ws[dev];
    if (!w) {
        w.reset(new Workspace());
        w->device = dev;
    }
    return *w;
}

template <typename T>
T *need(Workspace &ws, const char *name, size_t n, cudaStream_t st, bool keep = false)
{
    Buf &b = ws.bufs[name];
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    if (bytes > b.bytes) {
        size_t nb = std::max(bytes, b.bytes + b.bytes / 2);
        nb = (nb + 255) & ~(size_t)255;
        void *np = nullptr;
        cudaError_t e = cudaMalloc(&np, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{FMM_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(nb) +
                                           ") for " + name + ": " + cudaGetErrorString(e)};
        }
        if (keep && b.p) FMM_CUDA_TRY(cudaMemcpyAsync(np, b.p, b.bytes, cudaMemcpyDeviceToDevice, st));
        if (b.p) {
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            FMM_CUDA_TRY(cudaFree(b.p));
        }
        b.p = np;
        b.bytes = nb;
    }
    return static_cast<T *>(b.p);
}

void ensure_streams(Workspace &ws)
{
    if (ws.main_stream) return;
    int lo = 0, hi = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    FMM_CUDA_TRY(cudaStreamCreateWithFlags(&ws.main_stream, cudaStreamNonBlocking));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&ws.far_stream, cudaStreamNonBlocking, hi));
    for (cudaEvent_t *e : {&ws.ev_in, &ws.ev_tree, &ws.ev_fork, &ws.ev_join, &ws.ev_out, &ws.ev_read})
        FMM_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
}

template <typename T>
T *get(Workspace &ws, const char *name)
{
    return static_cast<T *>(ws.bufs[name].p);
}

void *pinned(Workspace &ws, size_t bytes)
{
    if (bytes > ws.pinned_bytes) {
        if (ws.pinned) cudaFreeHost(ws.pinned);
        ws.pinned = nullptr;
        size_t nb = std::max<size_t>(bytes, 4096);
        if (cudaMallocHost(&ws.pinned, nb) != cudaSuccess) {
            cudaGetLastError();
            ws.pinned_bytes = 0;
            throw Error{FMM_ERR_NOMEM, "cudaMallocHost failed"};
        }
        ws.pinned_bytes = nb;
    }
    return ws.pinned;
}

// Asynchronous upload through the pinned arena (no pageable copies, which can
// serialise with other streams).  The arena is reset at the start of a solve;
// every solve ends synchronised, so no upload of the previous one is in flight.
void upload(Workspace &ws, void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return;
    const size_t need_bytes = ws.up_off + ((bytes + 255) & ~(size_t)255);
    if (need_bytes > ws.up_bytes) {
        FMM_CUDA_TRY(cudaDeviceSynchronize());
        unsigned char *old = ws.up;
        const size_t nb = std::max<size_t>(need_bytes * 2, 1 << 20);
        if (cudaMallocHost(reinterpret_cast<void **>(&ws.up), nb) != cudaSuccess) {
            cudaGetLastError();
            ws.up = old;
            throw Error{FMM_ERR_NOMEM, "cudaMallocHost failed"};
        }
        if (old) cudaFreeHost(old);
        ws.up_bytes = nb;
        ws.up_off = 0;  // earlier uploads of this solve have completed (device synchronised)
    }
    unsigned char *h = ws.up + ws.up_off;
    std::memcpy(h, src, bytes);
    FMM_CUDA_TRY(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, st));
    ws.up_off += (bytes + 255) & ~(size_t)255;
}

// Copies the device flags plus `n` extra (dev -> host) items and synchronises.
// A read-back of the device flags and some device values, in two halves:
// read_begin enqueues the copies on st and records an event; read_end waits for
// that event only (work enqueued on st after read_begin keeps running), raises
// the error a flag reports and copies the values out.
struct ReadBack {
    char *h;
    size_t total;
};

ReadBack read_begin(Workspace &ws, cudaStream_t st, const int *flags_dev,
                    std::initializer_list<std::pair<const void *, size_t>> items)
{
    size_t total = sizeof(int) * kNumFlags;
    for (auto &it : items) total += it.second;
    char *h = static_cast<char *>(pinned(ws, total));
    FMM_CUDA_TRY(cudaMemcpyAsync(h, flags_dev, sizeof(int) * kNumFlags, cudaMemcpyDeviceToHost, st));
    size_t off = sizeof(int) * kNumFlags;
    for (auto &it : items) {
        FMM_CUDA_TRY(cudaMemcpyAsync(h + off, it.first, it.second, cudaMemcpyDeviceToHost, st));
        off += it.second;
    }
    if (!ws.ev_read) FMM_CUDA_TRY(cudaEventCreateWithFlags(&ws.ev_read, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventRecord(ws.ev_read, st));
    return {h, total};
}

void read_end(Workspace &ws, const ReadBack &rb, void *host_out)
{
    FMM_CUDA_TRY(cudaEventSynchronize(ws.ev_read));
    const int *f = reinterpret_cast<const int *>(rb.h);
    if (f[kFlagNonfinite]) throw Error{FMM_ERR_NONFINITE, "a coordinate is NaN or infinite"};
    if (f[kFlagHashFull]) throw Error{FMM_ERR_CAPACITY, "offset-class table is full"};
    if (f[kFlagClassRange])
        throw Error{FMM_ERR_CAPACITY, "an M2L offset exceeds the class key range (2^18 cells)"};
    if (f[kFlagStack]) throw Error{FMM_ERR_CAPACITY, "traversal stack overflow"};
    if (f[kFlagTimeout]) throw Error{FMM_ERR_TIMEOUT, "a bounded device-side wait expired (M2L pipeline)"};
    if (host_out) std::memcpy(host_out, rb.h + sizeof(int) * kNumFlags, rb.total - sizeof(int) * kNumFlags);
}

// Both halves at once: the host waits until st has reached the read-back.
void sync_point(Workspace &ws, cudaStream_t st, const int *flags_dev,
                std::initializer_list<std::pair<const void *, size_t>> items, void *host_out)
{
    read_end(ws, read_begin(ws, st, flags_dev, items), host_out);
}

struct Events {
    bool on = false;
    cudaEvent_t ev[11] = {};
    void init(bool enable)
    {
        on = enable;
        if (on)
            for (auto &e : ev) FMM_CUDA_TRY(cudaEventCreate(&e));
    }
    void rec(int i, cudaStream_t st)
    {
        if (on) FMM_CUDA_TRY(cudaEventRecord(ev[i], st));
    }
    float ms(int a, int b)
    {
        float v = 0.f;
        if (on) FMM_CUDA_TRY(cudaEventElapsedTime(&v, ev[a], ev[b]));
        return v;
    }
    ~Events()
    {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

__global__ void k_p2p_interactions(const int *__restrict__ tgt, const int *__restrict__ src,
                                   int64_t n, CellArrays c, unsigned long long *out)
{
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int t = tgt[i], so = src[i];
        s += (unsigned long long)(c.end[t] - c.begin[t]) * (unsigned long long)(c.end[so] - c.begin[so]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 16)
{
    int64_t g = ceil_div(std::max<int64_t>(n, 1), threads);
    return (unsigned)std::min(g, cap);
}

void validate(const void *xyz, const void *q, int64_t N, int p, double theta, int ncrit,
              const void *phi, const void *grad, const fmm_options &o)
{
    if (!xyz || !q || !phi || !grad) throw Error{FMM_ERR_ARG, "null pointer argument"};
    if (N < 1 || N >= (int64_t(1) << 31)) throw Error{FMM_ERR_ARG, "N must be in [1, 2^31)"};
    if (p < 1 || p > 20) throw Error{FMM_ERR_ARG, "p must be in [1, 20]"};
    if (!(theta > 0.0 && theta < 1.0)) throw Error{FMM_ERR_ARG, "theta must be in (0, 1)"};
    if (ncrit < 1) throw Error{FMM_ERR_ARG, "ncrit must be >= 1"};
    if (o.max_depth < 0 || o.max_depth > kMaxLevel) throw Error{FMM_ERR_ARG, "max_depth must be in [0, 21]"};
    if (o.precision_mode < FMM_PREC_FP32 || o.precision_mode > FMM_PREC_BF16X3)
        throw Error{FMM_ERR_ARG, "precision_mode must be FMM_PREC_FP32, _TF32X3 or _BF16X3"};
    if (o.select_mode < FMM_SELECT_PLAIN || o.select_mode > FMM_SELECT_TREECODE)
        throw Error{FMM_ERR_ARG, "select_mode must be one of FMM_SELECT_*"};
    if (o.m2l_unit_blocks < 0) throw Error{FMM_ERR_ARG, "m2l_unit_blocks must be >= 0"};
    if (o.select_mode == FMM_SELECT_TABLE && !o.select_table)
        throw Error{FMM_ERR_ARG, "FMM_SELECT_TABLE needs fmm_options.select_table"};

}

// The solve on device buffers; the caller holds ws.mu.
// lists_only: stop after the traversal (the tree, the leaves and the interaction
// lists stay in the workspace; phi and grad are not written).  blocks_only: go on
// to the offset classes and the M2L tiles and stop once the number of (tile,
// class) blocks is known (ws.shape.nent); no operator is built, nothing is
// evaluated.
void solve_locked(Workspace &ws, const float *xyz, const float *q, int64_t N64, int nsys,
                  const int64_t *offsets, int p, double theta, int ncrit, float *phi, float *grad,
                  cudaStream_t caller, const fmm_options &o, fmm_stats *stats, const uint8_t *sel,
                  bool lists_only = false, bool blocks_only = false)
{
    const bool no_eval = lists_only || blocks_only;
    ensure_streams(ws);
    init_recurrence_tables();
    cudaStream_t st = ws.main_stream;
    FMM_CUDA_TRY(cudaEventRecord(ws.ev_in, caller));
    FMM_CUDA_TRY(cudaStreamWaitEvent(st, ws.ev_in, 0));
    const int N = (int)N64;
    const int max_depth = o.max_depth == 0 ? kMaxLevel : o.max_depth;
    const int P2 = nterms(p), P2pad = nterms_pad(p);
    Events ev;
    ev.init(stats != nullptr);
    ws.have_solve = false;
    ws.up_off = 0;
    g_launch_count = 0;
    ev.rec(0, st);

    // ---------------------------------------------------------- box, keys, sort
    int *flags = need<int>(ws, "flags", kNumFlags, st);
    uint32_t *bbox_u = need<uint32_t>(ws, "bbox_u", 6 * (size_t)nsys, st);
    double *box = need<double>(ws, "box", 4 * (size_t)nsys, st);
    int *sys_off = need<int>(ws, "sys_off", nsys + 1, st);
    uint64_t *keys = need<uint64_t>(ws, "keys", N, st);
    uint64_t *keys_alt = need<uint64_t>(ws, "keys_alt", N, st);
    uint32_t *idx = need<uint32_t>(ws, "idx", N, st);
    uint32_t *idx_alt = need<uint32_t>(ws, "idx_alt", N, st);
    const int64_t nh = radix_scratch_elems(N);
    uint32_t *hist = need<uint32_t>(ws, "hist", nh, st);
    float4 *pts = need<float4>(ws, "pts", N, st);
    {
        std::vector<int> off32(nsys + 1);
        for (int sy = 0; sy <= nsys; ++sy) off32[sy] = (int)offsets[sy];
        upload(ws, sys_off, off32.data(), sizeof(int) * (nsys + 1), st);
    }
    FMM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * kNumFlags, st));
    k_init_bbox<<<(unsigned)ceil_div(6 * (int64_t)nsys, 256), 256, 0, st>>>(bbox_u, nsys);
    FMM_LAUNCH_CHECK();
    if (nsys == 1)
        k_bbox<<<grid_for(N, 256), 256, 0, st>>>(xyz, N, bbox_u, flags);
    else
        k_bbox_sys<<<(unsigned)ceil_div(ceil_div(N, 8), 256), 256, 0, st>>>(xyz, N, sys_off, nsys, bbox_u, flags);
    FMM_LAUNCH_CHECK();
    k_morton<<<grid_for(N, 256), 256, 0, st>>>(xyz, N, sys_off, nsys, bbox_u, box, keys, idx);
    FMM_LAUNCH_CHECK();
    if (nsys == 1) {
        radix_sort_pairs(keys, idx, keys_alt, idx_alt, N, 63, hist, flags, st);
    } else {
        // sort by key, then stably by system; the keys follow the permutation
        uint64_t *keys_orig = need<uint64_t>(ws, "keys_orig", N, st);
        uint64_t *sys_key = need<uint64_t>(ws, "sys_key", N, st);
        FMM_CUDA_TRY(cudaMemcpyAsync(keys_orig, keys, sizeof(uint64_t) * N, cudaMemcpyDeviceToDevice, st));
        radix_sort_pairs(keys, idx, keys_alt, idx_alt, N, 63, hist, flags, st);
        k_sys_of_sorted<<<grid_for(N, 256), 256, 0, st>>>(idx, N, sys_off, nsys, sys_key);
        FMM_LAUNCH_CHECK();
        int bits = 1;
        while ((1 << bits) < nsys) ++bits;
        radix_sort_pairs(sys_key, idx, keys_alt, idx_alt, N, bits, hist, flags, st);
        k_gather_keys<<<grid_for(N, 256), 256, 0, st>>>(keys_orig, idx, N, keys);
        FMM_LAUNCH_CHECK();
    }
    k_permute<<<grid_for(N, 256), 256, 0, st>>>(xyz, q, idx, N, pts);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- tree
    // When the previous solve had the same N, systems, ncrit and depth limit, its
    // level sizes (+50 %) serve as capacities: the levels are built with their
    // ranges kept on the device and the tree is read back once.  A tree that
    // outgrows them is rebuilt level by level with one read-back per level.
    const Workspace::Shape prev = ws.shape;
    const bool fast_tree = !prev.lstart.empty() && prev.N == N && prev.nsys == nsys && prev.ncrit == ncrit &&
                           prev.max_depth == max_depth;
    int cell_cap = std::max(1024, N / 8 + 64 + nsys);
    if (fast_tree) cell_cap = std::max<int64_t>(cell_cap, (int64_t)prev.ncells + prev.ncells / 2 + 1024 + nsys);
    auto cells = [&](int cap, bool keep) {
        CellArrays c;
        c.level = need<int>(ws, "c_level", cap, st, keep);
        c.prefix = need<uint64_t>(ws, "c_prefix", cap, st, keep);
        c.begin = need<int>(ws, "c_begin", cap, st, keep);
        c.end = need<int>(ws, "c_end", cap, st, keep);
        c.parent = need<int>(ws, "c_parent", cap, st, keep);
        c.child0 = need<int>(ws, "c_child0", cap, st, keep);
        c.nchild = need<int>(ws, "c_nchild", cap, st, keep);
        c.tile = need<int>(ws, "c_tile", cap, st, keep);
        c.lane = need<int>(ws, "c_lane", cap, st, keep);
        c.sys = need<int>(ws, "c_sys", cap, st, keep);
        c.geom = need<int4>(ws, "c_geom", cap, st, keep);
        c.fhi = need<float4>(ws, "c_fhi", cap, st, keep);
        c.flo = need<float4>(ws, "c_flo", cap, st, keep);
        return c;
    };
    CellArrays c = cells(cell_cap, false);
    k_init_roots<<<(unsigned)ceil_div(nsys, 256), 256, 0, st>>>(c, sys_off, nsys);
    FMM_LAUNCH_CHECK();
    // boundary positions of adjacent keys, bucketed (stably) by the level at which they differ
    uint64_t *blvl = need<uint64_t>(ws, "blvl", std::max(N - 1, 1), st);
    uint32_t *bpos = need<uint32_t>(ws, "bpos", std::max(N - 1, 1), st);
    int *bstart = need<int>(ws, "bstart", 24, st);
    if (N > 1) {
        k_first_diff<<<grid_for(N, 256), 256, 0, st>>>(keys, N, blvl, bpos);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(blvl, bpos, keys_alt, idx_alt, N - 1, 8, hist, flags, st);
    }
    k_level_starts<<<1, 32 * kLevelStartWarps, 0, st>>>(blvl, N - 1, bstart);
    FMM_LAUNCH_CHECK();
    std::vector<int> lstart;
    int tiles_total = 0;
    int nleaves = 0;
    int *leaves = nullptr;
    int *pcell = need<int>(ws, "pcell", std::max(N, 1), st);  // the leaf of each sorted particle
    bool tree_done = false;
    if (fast_tree) {
        const int pdepth = (int)prev.lstart.size() - 2;
        const int levels = std::min(pdepth + 1, max_depth);
        std::vector<int> cap(levels + 2, 0);
        for (int l = 0; l <= levels; ++l) {
            const int ll = std::min(l, pdepth);
            const int64_t cnt = prev.lstart[ll + 1] - prev.lstart[ll];
            cap[l] = (int)std::min<int64_t>(cnt + cnt / 2 + 256, cell_cap);
        }
        const int maxcap = *std::max_element(cap.begin(), cap.end());
        int *sz = need<int>(ws, "tree_sz", kSzWords, st);
        int64_t *packed = need<int64_t>(ws, "packed", maxcap + 1, st);
        int64_t *packed_ex = need<int64_t>(ws, "packed_ex", maxcap + 1, st);
        int64_t *i64_tmp = need<int64_t>(ws, "scan_i64", scan_temp_elems(std::max(maxcap, 1 << 16)), st);
        k_plan_init<<<1, 64, 0, st>>>(sz, nsys);
        FMM_LAUNCH_CHECK();
        // the first levels whose capacities are small: one block splits them all
        int nsmall = 0;
        while (nsmall < kMaxSmallLevels && nsmall <= levels && cap[nsmall] <= kSmallLevelCells) ++nsmall;
        if (nsmall > 0) {
            SmallLevels sl{};
            sl.n = nsmall;
            for (int l = 0; l <= nsmall; ++l) sl.cap[l] = cap[l];
            k_tree_small_levels<<<1, kSmallLevelThreads, 0, st>>>(c, keys, bpos, bstart, ncrit, max_depth, sl,
                                                                    levels, cell_cap, INT_MAX, sz);
            FMM_LAUNCH_CHECK();
        }
        for (int l = nsmall; l <= levels; ++l) {
            const int len = cap[l];
            k_split_count<<<(unsigned)ceil_div(len, 128), 128, 0, st>>>(c, bpos, bstart, 0, 0, l, ncrit, max_depth,
                                                                       packed, sz, len);
            FMM_LAUNCH_CHECK();
            scan_exclusive<int64_t>(packed, packed_ex, len, packed_ex + len, i64_tmp, st);
            k_level_advance<<<1, 1, 0, st>>>(packed_ex + len, l, levels, cell_cap, cap[l + 1], INT_MAX, sz);
            FMM_LAUNCH_CHECK();
            k_split_emit<<<(unsigned)ceil_div(len, 128), 128, 0, st>>>(c, keys, bpos, bstart, 0, 0, l, packed,
                                                                      packed_ex, 0, sz);
            FMM_LAUNCH_CHECK();
        }
        int *lflag = need<int>(ws, "leaf_flag", cell_cap, st);
        int *lex = need<int>(ws, "leaf_ex", cell_cap + 1, st);
        int *i32_tmp = need<int>(ws, "scan_i32", scan_temp_elems(cell_cap), st);
        leaves = need<int>(ws, "leaves", cell_cap, st);
        k_leaf_flags<<<(unsigned)ceil_div(cell_cap, 256), 256, 0, st>>>(c, 0, lflag, sz, cell_cap);
        FMM_LAUNCH_CHECK();
        scan_exclusive<int>(lflag, lex, cell_cap, lex + cell_cap, i32_tmp, st);
        k_leaf_compact<<<(unsigned)ceil_div(cell_cap, 256), 256, 0, st>>>(c, 0, lex, leaves, sz, pcell);
        FMM_LAUNCH_CHECK();
        FMM_CUDA_TRY(cudaMemcpyAsync(sz + kSzLeaves, lex + cell_cap, sizeof(int), cudaMemcpyDeviceToDevice, st));
        int hsz[kSzWords];
        sync_point(ws, st, flags, {{sz, sizeof(hsz)}}, hsz);
        if (!hsz[kSzAbort]) {
            lstart.push_back(hsz[kSzLevel]);
            for (int l = 0; l <= levels && hsz[kSzLevel + l + 1] > hsz[kSzLevel + l]; ++l)
                lstart.push_back(hsz[kSzLevel + l + 1]);
            tiles_total = hsz[kSzTiles];
            nleaves = hsz[kSzLeaves];
            tree_done = true;
        } else {
            k_init_roots<<<(unsigned)ceil_div(nsys, 256), 256, 0, st>>>(c, sys_off, nsys);
            FMM_LAUNCH_CHECK();
        }
    }
    if (!tree_done) {
        lstart = {0, nsys};
        tiles_total = (int)ceil_div(nsys, kTile);  // the roots' tiles
        int64_t *i64_tmp = need<int64_t>(ws, "scan_i64", scan_temp_elems(std::max(N, 1 << 16)), st);
        for (int l = 0;; ++l) {
            const int a = lstart[l], b = lstart[l + 1];
            const int nl = b - a;
            if (nl == 0) break;
            int64_t *packed = need<int64_t>(ws, "packed", nl, st);
            int64_t *packed_ex = need<int64_t>(ws, "packed_ex", nl + 1, st);
            i64_tmp = need<int64_t>(ws, "scan_i64", scan_temp_elems(nl), st);
            k_split_count<<<(unsigned)ceil_div(nl, 128), 128, 0, st>>>(c, bpos, bstart, a, b, l, ncrit,
                                                                      max_depth, packed);
            FMM_LAUNCH_CHECK();
            scan_exclusive<int64_t>(packed, packed_ex, nl, packed_ex + nl, i64_tmp, st);
            int64_t total = 0;
            sync_point(ws, st, flags, {{packed_ex + nl, sizeof(int64_t)}}, &total);
            const int nch = (int)(total & 0xffffffffll);
            const int nsplit = (int)(total >> 32);
            if (nch == 0) break;
            if (b + nch > cell_cap) {
                cell_cap = std::max(b + nch, cell_cap + cell_cap / 2);
                c = cells(cell_cap, true);
            }
            k_split_emit<<<(unsigned)ceil_div(nl, 128), 128, 0, st>>>(c, keys, bpos, bstart, a, b, l, packed,
                                                                     packed_ex, tiles_total);
            FMM_LAUNCH_CHECK();
            tiles_total += 8 * (int)ceil_div(nsplit, kTile);
            lstart.push_back(b + nch);
        }
    }
    const int depth = (int)lstart.size() - 2;
    const int ncells = lstart.back();
    if (!tree_done) {
        int *lflag = need<int>(ws, "leaf_flag", ncells, st);
        int *lex = need<int>(ws, "leaf_ex", ncells + 1, st);
        int *i32_tmp = need<int>(ws, "scan_i32", scan_temp_elems(ncells), st);
        leaves = need<int>(ws, "leaves", ncells, st);
        k_leaf_flags<<<(unsigned)ceil_div(ncells, 256), 256, 0, st>>>(c, ncells, lflag);
        FMM_LAUNCH_CHECK();
        scan_exclusive<int>(lflag, lex, ncells, lex + ncells, i32_tmp, st);
        k_leaf_compact<<<(unsigned)ceil_div(ncells, 256), 256, 0, st>>>(c, ncells, lex, leaves, nullptr, pcell);
        FMM_LAUNCH_CHECK();
        sync_point(ws, st, flags, {{lex + ncells, sizeof(int)}}, &nleaves);
    }
    k_cell_geom<<<grid_for(ncells, 256), 256, 0, st>>>(c, ncells, box);
    FMM_LAUNCH_CHECK();
    ev.rec(1, st);

    // ---------------------------------------------------------- upward pass (beside the traversal)
    // P2M and M2M need only the tree: they run on the far-field stream while the
    // traversal runs on the main stream.
    cudaStream_t fs = ws.far_stream;
    float *M = nullptr, *Lx = nullptr;
    if (!no_eval) {
        FMM_CUDA_TRY(cudaEventRecord(ws.ev_tree, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(fs, ws.ev_tree, 0));
        if (ws.cache_p != p) {
            // operator tables: shift matrices per p; the M2L matrices are cached per class key
            ws.class_cache.clear();
            ws.table_slots = 0;
            ws.split_slots = 0;
            ws.cache_p = p;
            float *m2m = need<float>(ws, "m2m", (size_t)8 * P2pad * P2pad, fs);
            float *l2l = need<float>(ws, "l2l", (size_t)8 * P2pad * P2pad, fs);
            double *m2m64 = nullptr, *l2l64 = nullptr;  // FP64 copies for the top levels at high p
            if (p >= kFp64TopP) {
                m2m64 = need<double>(ws, "m2m64", (size_t)8 * P2pad * P2pad, fs);
                l2l64 = need<double>(ws, "l2l64", (size_t)8 * P2pad * P2pad, fs);
            }
            const size_t sh = sizeof(double) * 2 * (size_t)(p + 1) * (p + 2) / 2;
            k_build_shift_tables<<<16, 256, sh, fs>>>(p, P2pad, m2m, l2l, m2m64, l2l64);
            FMM_LAUNCH_CHECK();
        }
        M = need<float>(ws, "M", (size_t)ncells * P2pad, fs);
        Lx = need<float>(ws, "L", (size_t)ncells * P2pad, fs);
        ev.rec(2, fs);
        launch_p2m(c, leaves, nleaves, (unsigned)nleaves, pts, p, P2pad, M, fs);
        float *mtmp = need<float>(ws, "m2m_tmp", (size_t)ncells * P2pad, fs);
        for (int l = depth - 1; l >= 0; --l) {
            const int a = lstart[l], b = lstart[l + 1];
            if (p >= kFp64TopP && l < kFp64TopLevels)
                launch_shift_fp64(false, c, a, b, get<double>(ws, "m2m64"), P2, P2pad, M, fs);
            else
                launch_shift_batched(false, c, a, b, get<float>(ws, "m2m"), P2, P2pad, M, mtmp, fs);
        }
        ev.rec(7, fs);
    }
    ws.shape.lstart = lstart;
    ws.shape.N = N;
    ws.shape.nsys = nsys;
    ws.shape.ncrit = ncrit;
    ws.shape.max_depth = max_depth;
    ws.shape.ncells = ncells;
    ws.shape.nleaves = nleaves;

    // ---------------------------------------------------------- traversal
    const double theta2 = theta * theta;
    ListArrays L;
    L.m2l_off = need<int>(ws, "m2l_off", ncells, st);
    L.m2l_cnt = need<int>(ws, "m2l_cnt", ncells, st);
    L.p2p_off = need<int>(ws, "p2p_off", ncells, st);
    L.p2p_cnt = need<int>(ws, "p2p_cnt", ncells, st);
    L.def_off = need<int>(ws, "def_off", ncells, st);
    L.def_cnt = need<int>(ws, "def_cnt", ncells, st);
    // capacities: the last solve's totals, or estimates; regrown exactly on overflow
    int64_t m2l_cap = std::max<int64_t>(ws.cap_m2l, std::max<int64_t>(4096, (int64_t)ncells * 160));
    int64_t p2p_cap = std::max<int64_t>(ws.cap_p2p, std::max<int64_t>(4096 + nsys, (int64_t)nleaves * 96));
    int64_t def_cap = std::max<int64_t>(ws.cap_def, std::max<int64_t>(4096 + nsys, (int64_t)ncells * 96));
    uint64_t *hash_keys = need<uint64_t>(ws, "hash_keys", kHashCap, st);
    unsigned long long *tcount = need<unsigned long long>(ws, "trav_counters", 5, st);
    // hybrid selection table (the flagged deferred sources need cell ids below 2^30)
    const uint8_t *d_sel = nullptr;
    ws.sel_host.assign((size_t)kSelNB * kSelNB, 0);
    if (sel) {
        if (ncells >= (1 << 29)) throw Error{FMM_ERR_CAPACITY, "selection tables need fewer than 2^29 cells"};
        std::memcpy(ws.sel_host.data(), sel, ws.sel_host.size());
        uint8_t *dsel = need<uint8_t>(ws, "select_table", ws.sel_host.size(), st);
        upload(ws, dsel, ws.sel_host.data(), ws.sel_host.size(), st);
        d_sel = dsel;
    }
    L.m2p_off = need<int>(ws, "m2p_off", ncells, st);
    L.m2p_cnt = need<int>(ws, "m2p_cnt", ncells, st);
    L.p2l_off = need<int>(ws, "p2l_off", ncells, st);
    L.p2l_cnt = need<int>(ws, "p2l_cnt", ncells, st);
    int64_t m2p_cap = std::max<int64_t>(ws.cap_m2p, 4096), p2l_cap = std::max<int64_t>(ws.cap_p2l, 4096);
    int64_t m2l_total = 0, p2p_total = 0, m2p_total = 0, p2l_total = 0;
    float4 *far = no_eval ? nullptr : need<float4>(ws, "far", N, st);
    float4 *near = no_eval ? nullptr : need<float4>(ws, "near", N, st);
    for (int attempt = 0;; ++attempt) {
        L.m2p_src = need<int>(ws, "m2p_src", m2p_cap, st);
        L.m2p_tgt = need<int>(ws, "m2p_tgt", m2p_cap, st);
        L.p2l_src = need<int>(ws, "p2l_src", p2l_cap, st);
        L.p2l_tgt = need<int>(ws, "p2l_tgt", p2l_cap, st);
        L.m2l_src = need<int>(ws, "m2l_src", m2l_cap, st);
        L.m2l_tgt = need<int>(ws, "m2l_tgt", m2l_cap, st);
        L.m2l_slot = need<uint32_t>(ws, "m2l_slot", m2l_cap, st);
        L.p2p_src = need<int>(ws, "p2p_src", p2p_cap, st);
        L.p2p_tgt = need<int>(ws, "p2p_tgt", p2p_cap, st);
        L.def_src = need<int>(ws, "def_src", def_cap, st);
        FMM_CUDA_TRY(cudaMemsetAsync(hash_keys, 0xff, sizeof(uint64_t) * kHashCap, st));
        k_root_lists<<<1, 256, 0, st>>>(c, L, nsys, tcount);
        FMM_LAUNCH_CHECK();
        for (int l = 1; l <= depth; ++l) {
            const int a = lstart[l], b = lstart[l + 1];
            const unsigned blocks = (unsigned)ceil_div((int64_t)(b - a) * 32, 128);
            k_traverse_level<<<blocks, 128, 0, st>>>(c, L, a, b, theta2, (float)theta2, d_sel, tcount,
                                                     m2l_cap, p2p_cap, def_cap, m2p_cap, p2l_cap, hash_keys,
                                                     flags);
            FMM_LAUNCH_CHECK();
        }
        ev.rec(10, st);  // the lists of this attempt are complete
        unsigned long long tot[5];
        const ReadBack rb = read_begin(ws, st, flags, {{tcount, sizeof(tot)}});
        if (!lists_only) {
            // P2P needs only the per-leaf lists: it is enqueued behind the read-back
            // of the list totals, and the host waits for the read-back alone while
            // P2P runs.  (If a list outgrew its buffer, the traversal and P2P run
            // again.)
            FMM_CUDA_TRY(cudaEventRecord(ws.ev_fork, st));
            FMM_CUDA_TRY(cudaStreamWaitEvent(fs, ws.ev_fork, 0));
            if (!blocks_only) {
                set_carveout_once((const void *)k_p2p, cudaSharedmemCarveoutMaxShared);
                ev.rec(8, st);
                k_p2p<<<(unsigned)std::max(1, nleaves), 32, 0, st>>>(c, L, leaves, nleaves, pts, near);
                FMM_LAUNCH_CHECK();
                ev.rec(9, st);
            }
        }
        read_end(ws, rb, tot);
        if ((int64_t)tot[0] <= m2l_cap && (int64_t)tot[1] <= p2p_cap && (int64_t)tot[2] <= def_cap &&
            (int64_t)tot[3] <= m2p_cap && (int64_t)tot[4] <= p2l_cap) {
            m2l_total = (int64_t)tot[0];
            p2p_total = (int64_t)tot[1];
            m2p_total = (int64_t)tot[3];
            p2l_total = (int64_t)tot[4];
            for (int k = 0; k < 5; ++k) ws.shape.tot[k] = (int64_t)tot[k];
            break;
        }
        if (attempt >= 3) throw Error{FMM_ERR_CAPACITY, "interaction lists kept outgrowing their buffers"};
        // While the deferred list fitted, every total is exact and the overflowed lists get
        // exactly what they need; otherwise deeper levels were cut short, their totals are
        // lower bounds, and every list grows with a margin.
        const bool exact = (int64_t)tot[2] <= def_cap;
        int64_t *caps[5] = {&m2l_cap, &p2p_cap, &def_cap, &m2p_cap, &p2l_cap};
        for (int k = 0; k < 5; ++k) {
            const int64_t need_k = (int64_t)tot[k];
            if (exact) {
                if (need_k > *caps[k]) *caps[k] = need_k + need_k / 16;
            } else {
                *caps[k] = std::max<int64_t>(2 * *caps[k], need_k + need_k / 4);
            }
        }
    }
    ws.cap_m2l = m2l_cap;
    ws.cap_p2p = p2p_cap;
    ws.cap_def = def_cap;
    ws.cap_m2p = m2p_cap;
    ws.cap_p2l = p2l_cap;
    if (lists_only) {
        FMM_CUDA_TRY(cudaEventRecord(ws.ev_out, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(caller, ws.ev_out, 0));
        return;
    }

    // ---------------------------------------------------------- fork
    // P2P (launched in the traversal loop above) runs on the main stream while
    // the far-field chain (classes, tiles, M2L, downward pass) runs on the
    // library's high-priority stream; the two join before the final sum.  P2P:
    // one warp (block) per leaf with up to 128 registers a thread, 16 warps per
    // SM; the packed arithmetic keeps more interactions in flight than with more
    // warps of fewer registers (measured 1.68 ms at 80 registers and 24 warps,
    // 1.60 ms at 128 and 16, uniform 1M).  That fills the register file; as
    // blocks retire, the far-field stream (higher priority) gets SMs for its class
    // and tile kernels, and M2L starts on SMs that P2P has drained.  An SM's
    // L1/shared split can only change when the SM is idle; with the maximum shared
    // carveout the far-field kernels (up to ~200 KB of shared memory) can start
    // on SMs that run P2P blocks.
    if (o.serialize_phases) {  // the far-field chain after P2P (each phase timed alone)
        FMM_CUDA_TRY(cudaEventRecord(ws.ev_fork, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(fs, ws.ev_fork, 0));
    }

    // ---------------------------------------------------------- M2L tiles regrouped
    // each level's cells ordered by octant, face distances and M2L count, and cut
    // into tiles (k_tile_keys), for the tensor-core M2L, whose work units split a
    // tile's class blocks: the CUDA-core M2L runs one block per tile, and tiles
    // that gather the cells of most pairs would set its pace.  Enqueued before the
    // class read-backs.
    const bool tensor = o.precision_mode != FMM_PREC_FP32 && m2l_tc_supported(P2pad);
    if (tensor) {
        uint64_t *tkey = need<uint64_t>(ws, "tile_key", ncells, fs);
        uint64_t *tkey_alt = need<uint64_t>(ws, "tile_key_alt", ncells, fs);
        uint32_t *tval = need<uint32_t>(ws, "tile_val", ncells, fs);
        uint32_t *tval_alt = need<uint32_t>(ws, "tile_val_alt", ncells, fs);
        uint32_t *thist = need<uint32_t>(ws, "tile_hist", radix_scratch_elems(ncells), fs);
        int *tlstart = need<int>(ws, "tile_lstart", (int)lstart.size(), fs);
        upload(ws, tlstart, lstart.data(), sizeof(int) * lstart.size(), fs);
        k_tile_keys<<<grid_for(ncells, 256), 256, 0, fs>>>(c, ncells, L.m2l_cnt, ncells, tkey, tval);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(tkey, tval, tkey_alt, tval_alt, ncells, kTileSortBits, thist, flags, fs);
        k_tile_assign<<<grid_for(ncells, 256), 256, 0, fs>>>(tkey, tval, ncells, tlstart, tiles_total, c);
        FMM_LAUNCH_CHECK();
    }

    // ---------------------------------------------------------- offset classes
    int nclass = 0;
    {
        int *hflag = need<int>(ws, "hflag", kHashCap, fs);
        int *hex = need<int>(ws, "hex", kHashCap + 1, fs);
        int *i32_tmp = need<int>(ws, "scan_i32", scan_temp_elems(kHashCap), fs);
        k_hash_flags<<<kHashCap / 256, 256, 0, fs>>>(hash_keys, hflag);
        FMM_LAUNCH_CHECK();
        scan_exclusive<int>(hflag, hex, kHashCap, hex + kHashCap, i32_tmp, fs);
        sync_point(ws, fs, flags, {{hex + kHashCap, sizeof(int)}}, &nclass);
        uint64_t *ukeys = need<uint64_t>(ws, "ukeys", nclass, fs);
        uint64_t *ukeys_alt = need<uint64_t>(ws, "ukeys_alt", nclass, fs);
        uint32_t *uslot = need<uint32_t>(ws, "uslot", nclass, fs);
        uint32_t *uslot_alt = need<uint32_t>(ws, "uslot_alt", nclass, fs);
        int *slot_class = need<int>(ws, "slot_class", kHashCap, fs);
        k_hash_compact<<<kHashCap / 256, 256, 0, fs>>>(hash_keys, hex, ukeys, uslot);
        FMM_LAUNCH_CHECK();
        if (nclass > 0 && nclass <= 6144) {
            // few classes: rank sort, one thread per key (fewer launches than the radix sort)
            k_rank_classes<<<(unsigned)ceil_div(nclass, 128), 128, 0, fs>>>(ukeys, uslot, nclass, ukeys_alt,
                                                                           slot_class);
            FMM_LAUNCH_CHECK();
            std::swap(ukeys, ukeys_alt);
        } else if (nclass > 0) {
            const int64_t nh2 = radix_scratch_elems(nclass);
            uint32_t *h2 = need<uint32_t>(ws, "hist", std::max(nh, nh2), fs);
            radix_sort_pairs(ukeys, uslot, ukeys_alt, uslot_alt, nclass, 64, h2, flags, fs);
            k_slot_to_class<<<(unsigned)ceil_div(nclass, 256), 256, 0, fs>>>(uslot, nclass, slot_class);
            FMM_LAUNCH_CHECK();
        }
        if (nclass > 0) {
            if (m2l_total > 0) {
                k_m2l_class<<<grid_for(m2l_total, 256), 256, 0, fs>>>(L.m2l_slot, m2l_total, slot_class);
                FMM_LAUNCH_CHECK();
            }
        }
        if (!blocks_only) {  // (the block count needs class indices, not operators)
            std::vector<uint64_t> hkeys(nclass);
            if (nclass > 0) sync_point(ws, fs, flags, {{ukeys, sizeof(uint64_t) * nclass}}, hkeys.data());
            std::vector<int> cls_slot(nclass);
            std::vector<uint64_t> new_keys;
            std::vector<int> new_slots;
            for (int i = 0; i < nclass; ++i) {
                auto it = ws.class_cache.find(hkeys[i]);
                if (it == ws.class_cache.end()) {
                    const int s = ws.table_slots++;
                    ws.class_cache.emplace(hkeys[i], s);
                    new_keys.push_back(hkeys[i]);
                    new_slots.push_back(s);
                    cls_slot[i] = s;
                } else {
                    cls_slot[i] = it->second;
                }
            }
            need<float>(ws, "table", (size_t)std::max(ws.table_slots, 1) * P2pad * P2pad, fs, true);
            int *class_slot = need<int>(ws, "class_slot", nclass, fs);
            if (nclass > 0) upload(ws, class_slot, cls_slot.data(), sizeof(int) * nclass, fs);
            if (!new_keys.empty()) {
                const int nnew = (int)new_keys.size();
                uint64_t *nk = need<uint64_t>(ws, "new_keys", nnew, fs);
                int *ns = need<int>(ws, "new_slots", nnew, fs);
                upload(ws, nk, new_keys.data(), sizeof(uint64_t) * nnew, fs);
                upload(ws, ns, new_slots.data(), sizeof(int) * nnew, fs);
                const size_t sh = sizeof(double) * 2 * (size_t)(2 * p + 1) * (2 * p + 2) / 2;
                k_build_m2l_tables<<<nnew, 256, sh, fs>>>(nk, ns, nnew, p, P2pad, get<float>(ws, "table"));
                FMM_LAUNCH_CHECK();
            }
        }
    }

    // ---------------------------------------------------------- M2L tiles
    const int ntiles = tiles_total;
    const int nwords = std::max(1, (int)ceil_div(nclass, 32));
    int *tile_cells = need<int>(ws, "tile_cells", (size_t)ntiles * kTile, fs);
    uint32_t *bitmap = need<uint32_t>(ws, "bitmap", (size_t)ntiles * nwords, fs);
    int *tile_cnt = need<int>(ws, "tile_cnt", ntiles, fs);
    int *entry_base = need<int>(ws, "entry_base", ntiles + 1, fs);
    int *word_prefix = need<int>(ws, "word_prefix", (size_t)ntiles * nwords, fs);
    FMM_CUDA_TRY(cudaMemsetAsync(tile_cells, 0xff, sizeof(int) * (size_t)ntiles * kTile, fs));
    FMM_CUDA_TRY(cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * (size_t)ntiles * nwords, fs));
    k_fill_tile_cells<<<(unsigned)ceil_div(ncells, 256), 256, 0, fs>>>(c, ncells, tile_cells);
    FMM_LAUNCH_CHECK();
    if (m2l_total > 0) {
        k_tile_bitmap<<<grid_for(m2l_total, 256), 256, 0, fs>>>(L.m2l_tgt, L.m2l_slot, m2l_total,
                                                              c.tile, nwords, bitmap);
        FMM_LAUNCH_CHECK();
    }
    k_tile_popc<<<(unsigned)ceil_div(ntiles, 4), 128, 0, fs>>>(bitmap, ntiles, nwords, tile_cnt);
    FMM_LAUNCH_CHECK();
    {
        int *i32_tmp = need<int>(ws, "scan_i32", scan_temp_elems(ntiles), fs);
        scan_exclusive<int>(tile_cnt, entry_base, ntiles, entry_base + ntiles, i32_tmp, fs);
    }
    std::vector<int> h_eb(ntiles + 1);
    sync_point(ws, fs, flags, {{entry_base, sizeof(int) * (ntiles + 1)}}, h_eb.data());
    const int nent = h_eb[ntiles];
    ws.shape.nclass = nclass;
    ws.shape.ntiles = ntiles;
    ws.shape.nent = nent;
    ws.shape.nunits = 0;
    if (blocks_only) {
        FMM_CUDA_TRY(cudaEventRecord(ws.ev_out, fs));
        FMM_CUDA_TRY(cudaStreamWaitEvent(caller, ws.ev_out, 0));
        return;
    }
    int *entry_class = need<int>(ws, "entry_class", nent, fs);
    int *src = need<int>(ws, "src", (size_t)nent * kTile, fs);
    FMM_CUDA_TRY(cudaMemsetAsync(src, 0xff, sizeof(int) * (size_t)nent * kTile, fs));
    k_tile_entries<<<(unsigned)ceil_div(ntiles, 4), 128, 0, fs>>>(bitmap, ntiles, nwords, entry_base,
                                                                  word_prefix, entry_class,
                                                                  get<int>(ws, "class_slot"));
    FMM_LAUNCH_CHECK();
    if (m2l_total > 0) {
        k_tile_src_rows<<<(unsigned)ceil_div((int64_t)ntiles * kTile, 4), 128, 0, fs>>>(
            tile_cells, ntiles, L.m2l_off, L.m2l_cnt, L.m2l_src, L.m2l_slot, nwords, bitmap, word_prefix, src);
        FMM_LAUNCH_CHECK();
    }

    // ---------------------------------------------------------- M2L
    if (tensor) {
        // work units: (tile, contiguous run of its class blocks), about six per SM
        const int chunk = o.m2l_unit_blocks > 0 ? o.m2l_unit_blocks
                                                : std::max(8, (int)ceil_div(std::max(nent, 1), 6 * 152));
        // units in execution order: the full ones by (rank within the tile, tile), so that
        // resident CTAs work on similar class ranges, then each tile's shorter last unit by
        // size class, longer first (an SM takes the next unit as it frees, and short units
        // last even out the SMs' ends); tile_units lists each tile's units in class order
        // for the sum
        std::vector<int> nut(ntiles), ubase(ntiles + 1, 0);
        int maxr = 0;
        for (int t = 0; t < ntiles; ++t) {
            nut[t] = (int)ceil_div(h_eb[t + 1] - h_eb[t], chunk);
            ubase[t + 1] = ubase[t] + nut[t];
            maxr = std::max(maxr, nut[t]);
        }
        const int nunits = ubase[ntiles];
        ws.shape.nunits = nunits;
        ws.shape.chunk = chunk;
        std::vector<M2LUnit> units;
        units.reserve(nunits);
        std::vector<int> tile_units(std::max(nunits, 1));
        auto bucket = [&](int t, int r) {
            const int n = std::min(chunk, h_eb[t + 1] - (h_eb[t] + r * chunk));
            return n == chunk ? kUnitBuckets : n * kUnitBuckets / (chunk + 1);
        };
        auto place = [&](int t, int r) {
            const int e = h_eb[t] + r * chunk;
            tile_units[ubase[t] + r] = (int)units.size();
            units.push_back({t, e, std::min(e + chunk, h_eb[t + 1]), 0});
        };
        for (int r = 0; r < maxr; ++r)
            for (int t = 0; t < ntiles; ++t)
                if (r < nut[t] && bucket(t, r) == kUnitBuckets) place(t, r);
        for (int k = kUnitBuckets - 1; k >= 0; --k)
            for (int t = 0; t < ntiles; ++t)
                if (nut[t] > 0 && bucket(t, nut[t] - 1) == k) place(t, nut[t] - 1);
        M2LUnit *d_units = need<M2LUnit>(ws, "m2l_units", std::max(nunits, 1), fs);
        int *d_ubase = need<int>(ws, "m2l_ubase", ntiles + 1, fs);
        int *d_tunits = need<int>(ws, "m2l_tile_units", std::max(nunits, 1), fs);
        float *partial = need<float>(ws, "m2l_partial", (size_t)std::max(nunits, 1) * 128 * P2pad, fs);
        if (nunits > 0) {
            upload(ws, d_units, units.data(), sizeof(M2LUnit) * nunits, fs);
            upload(ws, d_tunits, tile_units.data(), sizeof(int) * nunits, fs);
        }
        upload(ws, d_ubase, ubase.data(), sizeof(int) * (ntiles + 1), fs);
        ev.rec(3, fs);
        // class matrices split into hi/lo in the stage layout, once per class slot and precision
        const bool bf16 = o.precision_mode == FMM_PREC_BF16X3;
        if (ws.split_prec != o.precision_mode) {
            ws.split_prec = o.precision_mode;
            ws.split_slots = 0;
        }
        unsigned char *tsplit = need<unsigned char>(ws, "table_split",
                                                    m2l_split_bytes(P2pad, bf16, std::max(ws.table_slots, 1)), fs, true);
        launch_split_tables(bf16, get<float>(ws, "table"), ws.split_slots, ws.table_slots - ws.split_slots, P2pad,
                            tsplit, fs);
        ws.split_slots = ws.table_slots;
        launch_m2l_tc(bf16, nunits, d_units, ntiles, d_ubase, d_tunits,
                      entry_class, src, tile_cells, M, tsplit, P2pad, partial, Lx,
                      flags, fs);
    } else {
        ev.rec(3, fs);
        launch_m2l_simt(ntiles, entry_base, entry_class, src, tile_cells, M, get<float>(ws, "table"),
                        P2pad, Lx, fs);
    }
    ev.rec(4, fs);

    // ---------------------------------------------------------- downward pass
    if (p2l_total > 0) {  // particle-cell pairs of the hybrid selection, into L before L2L
        const size_t sh = (size_t)32 * (P2pad + 1) * sizeof(float);
        if (sh > 48 * 1024) set_smem_limit_once((const void *)k_p2l, (int)sh);
        k_p2l<<<(unsigned)ncells, 32, sh, fs>>>(c, L, ncells, pts, box, p, P2pad, Lx);
        FMM_LAUNCH_CHECK();
    }
    for (int l = 0; l < depth; ++l)  // parents at level l, children at level l + 1
        if (p >= kFp64TopP && l < kFp64TopLevels)
            launch_shift_fp64(true, c, lstart[l], lstart[l + 1], get<double>(ws, "l2l64"), P2, P2pad, Lx, fs);
        else
            launch_shift_batched(true, c, lstart[l], lstart[l + 1], get<float>(ws, "l2l"), P2, P2pad, Lx, nullptr, fs);
    launch_l2p(c, pcell, N, pts, p, P2pad, Lx, far, fs);
    if (m2p_total > 0) {  // cell-particle pairs of the hybrid selection, added to the far field
        const size_t sh = m2p_smem(p, P2pad);
        if (sh > 48 * 1024) set_smem_limit_once((const void *)k_m2p, (int)sh);
        k_m2p<<<(unsigned)ceil_div(nleaves, kM2PWarps), 32 * kM2PWarps, sh, fs>>>(c, L, leaves, nleaves, pts, box, p,
                                                                                P2pad, M, far);
        FMM_LAUNCH_CHECK();
    }
    ev.rec(5, fs);

    // ---------------------------------------------------------- join and combine
    FMM_CUDA_TRY(cudaEventRecord(ws.ev_join, fs));
    FMM_CUDA_TRY(cudaStreamWaitEvent(st, ws.ev_join, 0));
    k_combine<<<grid_for(N, 256), 256, 0, st>>>(far, near, idx, N, phi, grad);
    FMM_LAUNCH_CHECK();
    ev.rec(6, st);

    unsigned long long *inter = nullptr;
    if (stats) {
        inter = need<unsigned long long>(ws, "inter", 1, st);
        FMM_CUDA_TRY(cudaMemsetAsync(inter, 0, sizeof(unsigned long long), st));
        if (p2p_total > 0) {
            k_p2p_interactions<<<grid_for(p2p_total, 256), 256, 0, st>>>(L.p2p_tgt, L.p2p_src,
                                                                       p2p_total, c, inter);
            FMM_LAUNCH_CHECK();
        }
    }
    unsigned long long ninter = 0;
    if (stats)
        sync_point(ws, st, flags, {{inter, sizeof(unsigned long long)}}, &ninter);
    else
        sync_point(ws, st, flags, {}, nullptr);
    FMM_CUDA_TRY(cudaEventRecord(ws.ev_out, st));
    FMM_CUDA_TRY(cudaStreamWaitEvent(caller, ws.ev_out, 0));

    ws.have_solve = true;
    ws.N = N;
    ws.nsys = nsys;
    ws.ncells = ncells;
    ws.nleaves = nleaves;
    ws.depth = depth;
    ws.P2pad = P2pad;
    ws.nclass = nclass;
    ws.nm2l = m2l_total;
    ws.np2p = p2p_total;
    ws.nm2p = m2p_total;
    ws.np2l = p2l_total;
    if (stats) {
        stats->n_m2p_pairs = m2p_total;
        stats->n_p2l_pairs = p2l_total;
        stats->ncells = ncells;
        stats->nleaves = nleaves;
        stats->depth = depth;
        stats->n_p2p_pairs = p2p_total;
        stats->n_p2p_interactions = (int64_t)ninter;
        stats->n_m2l_pairs = m2l_total;
        stats->n_offset_classes = nclass;
        stats->n_m2l_blocks = nent;
        stats->n_launches = g_launch_count - 1;  // minus the statistics kernel
        stats->ms_tree = ev.ms(0, 1);
        stats->ms_traverse = ev.ms(1, 10);  // the traversal alone (with its count read-backs)
        stats->ms_upward = ev.ms(2, 7);
        stats->ms_m2l = ev.ms(3, 4);  // the M2L kernel and its unit reduction only
        stats->ms_downward = ev.ms(4, 5);
        stats->ms_p2p = ev.ms(8, 9);  // P2P kernel alone (it overlaps the far-field chain)
        stats->ms_total = ev.ms(0, 6);
    }
}

// Time per M2L pair from plain solves of an artificial uniform cube (2^18
// particles, ncrit 32): M2L kernel time over the number of M2L pairs.
double m2l_ns_per_pair(Workspace &ws, int p, double theta, int prec)
{
    const auto key = std::make_tuple(p, (uint64_t)std::llround(theta * 1e9), prec);
    auto it = ws.m2l_ns.find(key);
    if (it != ws.m2l_ns.end()) return it->second;
    ensure_streams(ws);
    cudaStream_t st = ws.main_stream;
    const int64_t n = 1 << 18;
    float *xyz = need<float>(ws, "syn_xyz", 3 * n, st);
    float *q = need<float>(ws, "syn_q", n, st);
    float *phi = need<float>(ws, "syn_phi", n, st);
    float *grad = need<float>(ws, "syn_grad", 3 * n, st);
    synth_uniform(xyz, q, n, 0x5eed0001ull, st);
    fmm_options o;
    fmm_default_options(&o);
    o.precision_mode = prec;
    o.serialize_phases = 1;  // the M2L kernel's time alone
    const int64_t off[2] = {0, n};
    double best = 1e30;
    for (int rep = 0; rep < 3; ++rep) {
        fmm_stats s{};
        solve_locked(ws, xyz, q, n, 1, off, p, theta, 32, phi, grad, st, o, &s, nullptr);
        if (rep > 0 && s.n_m2l_pairs > 0) best = std::min(best, (double)s.ms_m2l * 1e6 / (double)s.n_m2l_pairs);
    }
    ws.have_solve = false;
    ws.m2l_ns[key] = best;
    return best;
}

// The parts of a solve's time that the N_crit pick does not take from the
// network, measured on an artificial clustered set (a Plummer sphere of 2^20
// particles) at N_crit 32 and 256, the range of the usual candidates (best of
// two repetitions each), each as a line through the two solves:
//  * the M2L kernel's time against its (tile, class) blocks -- the kernel's work
//    is per block, whatever the block's share of rows with a pair, so on a
//    clustered set or at a large N_crit the time per pair grows;
//  * the time outside the P2P and M2L kernels (tree levels, traversal, upward
//    and downward passes, class and tile building) against the cells, the part
//    that grows as N_crit shrinks.
SolveCal solve_calibration(Workspace &ws, int p, double theta, int prec)
{
    const auto key = std::make_tuple(p, (uint64_t)std::llround(theta * 1e9), prec);
    auto it = ws.cell_ns.find(key);
    if (it != ws.cell_ns.end()) return it->second;
    ensure_streams(ws);
    cudaStream_t st = ws.main_stream;
    const int64_t n = 1 << 20;
    float *xyz = need<float>(ws, "syn_xyz", 3 * n, st);
    float *q = need<float>(ws, "syn_q", n, st);
    float *phi = need<float>(ws, "syn_phi", n, st);
    float *grad = need<float>(ws, "syn_grad", 3 * n, st);
    synth_plummer(xyz, q, n, 0x5eed0005ull, st);
    fmm_options o;
    fmm_default_options(&o);
    o.precision_mode = prec;
    o.serialize_phases = 1;  // P2P and M2L each timed alone
    const int64_t off[2] = {0, n};
    double rest[2] = {1e30, 1e30}, m2l[2] = {1e30, 1e30}, cells[2] = {0, 0}, blocks[2] = {0, 0};
    const int ncs[2] = {32, 256};
    SolveCal c;
    unsigned long long *hist = need<unsigned long long>(ws, "pick_hist", (size_t)kSelNB * kSelNB, st);
    for (int k = 0; k < 2; ++k) {
        c.p2p_ns[k] = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            fmm_stats s{};
            solve_locked(ws, xyz, q, n, 1, off, p, theta, ncs[k], phi, grad, st, o, &s, nullptr);
            if (rep == 0) continue;  // warm-up (operator tables, buffers)
            rest[k] = std::min(rest[k], (double)(s.ms_total - s.ms_p2p - s.ms_m2l) * 1e6);
            m2l[k] = std::min(m2l[k], (double)s.ms_m2l * 1e6);
            c.p2p_ns[k] = std::min(c.p2p_ns[k], (double)s.ms_p2p * 1e6);
            cells[k] = (double)s.ncells;
            blocks[k] = (double)s.n_m2l_blocks;
        }
        // this solve's P2P pairs by count bucket
        const int64_t np2p = ws.shape.tot[1];
        FMM_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kSelNB * kSelNB, st));
        if (np2p > 0) {
            k_pair_bucket_hist<<<grid_for(np2p, 256), 256, 0, st>>>(get<int>(ws, "p2p_tgt"), get<int>(ws, "p2p_src"),
                                                                  np2p, get<int>(ws, "c_begin"), get<int>(ws, "c_end"),
                                                                  hist);
            FMM_LAUNCH_CHECK();
        }
        c.hist[k].resize((size_t)kSelNB * kSelNB);
        FMM_CUDA_TRY(cudaMemcpyAsync(c.hist[k].data(), hist, sizeof(unsigned long long) * kSelNB * kSelNB,
                                     cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ws.have_solve = false;
    // lines through the two solves (slopes kept >= 0)
    c.ns_block = blocks[0] > blocks[1] ? std::max(0.0, (m2l[0] - m2l[1]) / (blocks[0] - blocks[1])) : 0.0;
    c.ns_cell = cells[0] > cells[1] ? std::max(0.0, (rest[0] - rest[1]) / (cells[0] - cells[1])) : 0.0;
    c.ns_fixed = std::max(0.0, m2l[1] - c.ns_block * blocks[1]) + std::max(0.0, rest[1] - c.ns_cell * cells[1]);
    ws.cell_ns[key] = c;
    return c;
}

const std::vector<int> kSelCounts = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};

const std::vector<P2PTiming> &p2p_timings(Workspace &ws)
{
    if (ws.p2p_grid.empty()) {
        ensure_streams(ws);
        ws.p2p_grid = pretime_p2p(kSelCounts, 0x5eed0002ull, ws.main_stream);
    }
    return ws.p2p_grid;
}

const std::vector<double> &m2p_timings(Workspace &ws, int p)
{
    auto it = ws.m2p_ns.find(p);
    if (it != ws.m2p_ns.end()) return it->second;
    ensure_streams(ws);
    return ws.m2p_ns[p] = pretime_m2p(p, kSelCounts, 0x5eed0003ull, ws.main_stream);
}

const std::vector<double> &p2l_timings(Workspace &ws, int p)
{
    auto it = ws.p2l_ns.find(p);
    if (it != ws.p2l_ns.end()) return it->second;
    ensure_streams(ws);
    init_recurrence_tables();
    return ws.p2l_ns[p] = pretime_p2l(p, kSelCounts, 0x5eed0004ull, ws.main_stream);
}

const std::vector<uint8_t> &pretimed_table(Workspace &ws, int p, double theta, int prec)
{
    const auto key = std::make_tuple(FMM_SELECT_AUTOTUNE, (uint64_t)std::llround(theta * 1e9), p, prec);
    auto it = ws.tables.find(key);
    if (it != ws.tables.end()) return it->second;
    const double m2l = m2l_ns_per_pair(ws, p, theta, prec);
    std::vector<uint8_t> t((size_t)kSelNB * kSelNB);
    table_from_timings(p2p_timings(ws), m2l, kSelCounts, m2p_timings(ws, p), p2l_timings(ws, p), t.data());
    return ws.tables[key] = std::move(t);
}

const std::vector<uint8_t> &learned_table(Workspace &ws, int p, double theta)
{
    const auto key = std::make_tuple(FMM_SELECT_LEARNED, (uint64_t)std::llround(theta * 1e9), p, 0);
    auto it = ws.tables.find(key);
    if (it != ws.tables.end()) return it->second;
    ensure_streams(ws);
    std::vector<uint8_t> t((size_t)kSelNB * kSelNB);
    model_table(ws.cm, p, theta, t.data(), ws.main_stream);
    return ws.tables[key] = std::move(t);
}

// The selection table of a solve (nullptr = plain FMM).  Pre-timed tables are
// measured once per (p, theta, precision) and device; the learned mode falls
// back to them while no model has been trained or set.
const uint8_t *selection_table(Workspace &ws, const fmm_options &o, int p, double theta)
{
    switch (o.select_mode) {
        case FMM_SELECT_TABLE: return o.select_table;
        case FMM_SELECT_TREECODE: {
            static const std::vector<uint8_t> all_m2p((size_t)kSelNB * kSelNB, 2);
            return all_m2p.data();
        }
        case FMM_SELECT_AUTOTUNE: return pretimed_table(ws, p, theta, o.precision_mode).data();
        case FMM_SELECT_LEARNED:
            if (!ws.cm.trained) return pretimed_table(ws, p, theta, o.precision_mode).data();
            return learned_table(ws, p, theta).data();
        default: return nullptr;
    }
}

fmm_options resolve_opts(const fmm_options *opt)
{
    fmm_options o;
    fmm_default_options(&o);
    if (opt) o = *opt;
    return o;
}

Samples host_samples(const float *x, const float *t, const float *m, int64_t B)
{
    if (!x || B < 1) throw Error{FMM_ERR_ARG, "need x and B >= 1"};
    Samples s;
    s.x.assign(x, x + 4 * B);
    s.t.assign(2 * B, 0.f);
    s.m.assign(2 * B, 0.f);
    if (t) s.t.assign(t, t + 2 * B);
    if (m) s.m.assign(m, m + 2 * B);
    return s;
}

template <typename F>
fmm_status guarded(F &&f)
{
    try {
        f();
        set_last_error("");
        return FMM_OK;
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return FMM_ERR_NOMEM;
    } catch (...) {
        set_last_error("unexpected exception");
        return FMM_ERR_CUDA;
    }
}


// ---------------------------------------------------------------- captured plans

int64_t with_headroom(int64_t n, double h, int64_t margin) { return (int64_t)std::ceil((double)n * h) + margin; }

// Capacities of a plan from the sizes of its first solve.
PlanShape plan_shape(const Workspace &ws, int64_t N, int nsys, int p, double theta, int ncrit, const fmm_options &o,
                     bool hybrid, double h)
{
    const Workspace::Shape &sh = ws.shape;
    PlanShape s;
    s.N = (int)N;
    s.nsys = nsys;
    s.p = p;
    s.P2 = nterms(p);
    s.P2pad = nterms_pad(p);
    s.ncrit = ncrit;
    s.max_depth = o.max_depth == 0 ? kMaxLevel : o.max_depth;
    s.theta = theta;
    s.tensor = o.precision_mode != FMM_PREC_FP32 && m2l_tc_supported(s.P2pad);
    s.bf16 = o.precision_mode == FMM_PREC_BF16X3;
    s.hybrid = hybrid;
    s.sys_bits = 1;
    while ((1 << s.sys_bits) < nsys) ++s.sys_bits;
    const int depth = (int)sh.lstart.size() - 2;
    s.levels = std::min(depth + 1, s.max_depth);
    s.cell_cap = (int)std::min<int64_t>(with_headroom(sh.ncells, h, 1024 + nsys), INT_MAX / 2);
    s.level_cap.assign(s.levels + 2, 0);
    for (int l = 0; l <= s.levels; ++l) {
        const int cnt = l <= depth ? sh.lstart[l + 1] - sh.lstart[l] : sh.lstart[depth + 1] - sh.lstart[depth];
        s.level_cap[l] = (int)std::min<int64_t>(with_headroom(cnt, h, 256), s.cell_cap);
    }
    s.level_cap[s.levels + 1] = 0;  // the last level may not split
    s.max_level_cap = *std::max_element(s.level_cap.begin(), s.level_cap.end());
    s.leaf_cap = s.cell_cap;
    s.tile_cap = (int)with_headroom(sh.ntiles, h, 64);
    s.nclass_cap = (int)std::min<int64_t>(with_headroom(sh.nclass, h, 256), kHashCap);
    s.nwords = std::max(1, (int)ceil_div(s.nclass_cap, 32));
    s.nent_cap = (int)with_headroom(sh.nent, h, 1024);
    s.units_cap = (int)with_headroom(sh.nunits, h, 256);
    s.chunk = std::max(1, sh.chunk);
    s.m2l_cap = with_headroom(sh.tot[0], h, 4096);
    s.p2p_cap = with_headroom(sh.tot[1], h, 4096);
    s.def_cap = with_headroom(sh.tot[2], h, 4096);
    // A kind of pair the captured solve did not have gets no capacity and no kernel:
    // a replay whose lists hold one exceeds its capacity and is solved again plainly.
    s.m2p_seen = sh.tot[3] > 0;
    s.p2l_seen = sh.tot[4] > 0;
    s.m2p_cap = s.m2p_seen ? with_headroom(sh.tot[3], h, 4096) : 0;
    s.p2l_cap = s.p2l_seen ? with_headroom(sh.tot[4], h, 4096) : 0;
    s.class_hcap = 1;
    while (s.class_hcap < 2u * (uint32_t)std::max<int64_t>(1, (int64_t)ws.class_cache.size())) s.class_hcap <<= 1;
    int nsm = 152;
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws.device));
    s.nsm = nsm;
    return s;
}

}  // namespace
}  // namespace fmm

struct fmm_plan {
    int device = 0;
    fmm::PlanShape s;
    fmm::PlanBuffers b;
    fmm::PlanMemory mem;
    int64_t operators = 0, graph_nodes = 0, graph_kernels = 0;
    float *xyz = nullptr, *q = nullptr, *phi = nullptr, *grad = nullptr;
    cudaStream_t st = nullptr, fs = nullptr;
    cudaEvent_t tree = nullptr, fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int *hcheck = nullptr;  // pinned: the flags and sizes read back by a check
    fmm::IoPtrs *io = nullptr, *hio = nullptr;  // the caller's arrays of each replay (device, pinned host)
    ~fmm_plan()
    {
        if (st) cudaStreamSynchronize(st);
        if (hcheck) cudaFreeHost(hcheck);
        if (hio) cudaFreeHost(hio);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (tree) cudaEventDestroy(tree);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (st) cudaStreamDestroy(st);
        if (fs) cudaStreamDestroy(fs);
    }
};

namespace fmm {
namespace {

// Allocates the plan's buffers, copies the operators, and captures the graph.
void build_plan(fmm_plan &pl, Workspace &ws, const int64_t *offsets, const uint8_t *sel)
{
    const PlanShape &s = pl.s;
    PlanBuffers &b = pl.b;
    PlanMemory &m = pl.mem;
    const int N = s.N, nsys = s.nsys, P2pad = s.P2pad;
    const int64_t cc = s.cell_cap;
    FMM_CUDA_TRY(cudaStreamCreateWithFlags(&pl.st, cudaStreamNonBlocking));
    int lo = 0, hi = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&pl.fs, cudaStreamNonBlocking, hi));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&pl.tree, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&pl.fork, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&pl.join, cudaEventDisableTiming));

    b.xyz = pl.xyz;
    b.q = pl.q;
    b.phi = pl.phi;
    b.grad = pl.grad;
    b.io = pl.io;
    b.flags = m.get<int>(kNumFlags);
    b.sz = m.get<int>(kSzWords);
    b.bbox_u = m.get<uint32_t>(6 * (size_t)nsys);
    b.box = m.get<double>(4 * (size_t)nsys);
    b.sys_off = m.get<int>(nsys + 1);
    b.keys = m.get<uint64_t>(N);
    b.keys_alt = m.get<uint64_t>(N);
    b.idx = m.get<uint32_t>(N);
    b.idx_alt = m.get<uint32_t>(N);
    if (nsys > 1) {
        b.keys_orig = m.get<uint64_t>(N);
        b.sys_key = m.get<uint64_t>(N);
    }
    b.hist = m.get<uint32_t>(radix_scratch_elems(N));
    b.pts = m.get<float4>(N);
    b.c.level = m.get<int>(cc);
    b.c.prefix = m.get<uint64_t>(cc);
    b.c.begin = m.get<int>(cc);
    b.c.end = m.get<int>(cc);
    b.c.parent = m.get<int>(cc);
    b.c.child0 = m.get<int>(cc);
    b.c.nchild = m.get<int>(cc);
    b.c.tile = m.get<int>(cc);
    b.c.lane = m.get<int>(cc);
    b.c.sys = m.get<int>(cc);
    b.c.geom = m.get<int4>(cc);
    b.c.fhi = m.get<float4>(cc);
    b.c.flo = m.get<float4>(cc);
    b.blvl = m.get<uint64_t>(std::max(N - 1, 1));
    b.bpos = m.get<uint32_t>(std::max(N - 1, 1));
    b.bstart = m.get<int>(24);
    b.packed = m.get<int64_t>(s.max_level_cap + 1);
    b.packed_ex = m.get<int64_t>(s.max_level_cap + 1);
    b.scan_i64 = m.get<int64_t>(scan_temp_elems(s.max_level_cap));
    b.leaf_flag = m.get<int>(cc);
    b.leaf_ex = m.get<int>(cc + 1);
    b.scan_i32 = m.get<int>(scan_temp_elems(std::max<int64_t>({cc, (int64_t)kHashCap, (int64_t)s.tile_cap})));
    b.leaves = m.get<int>(cc);
    b.pcell = m.get<int>(std::max<int64_t>(s.N, 1));
    ListArrays &L = b.L;
    for (int **a : {&L.m2l_off, &L.m2l_cnt, &L.p2p_off, &L.p2p_cnt, &L.def_off, &L.def_cnt, &L.m2p_off, &L.m2p_cnt,
                    &L.p2l_off, &L.p2l_cnt})
        *a = m.get<int>(cc);
    L.m2l_src = m.get<int>(s.m2l_cap);
    L.m2l_tgt = m.get<int>(s.m2l_cap);
    L.m2l_slot = m.get<uint32_t>(s.m2l_cap);
    L.p2p_src = m.get<int>(s.p2p_cap);
    L.p2p_tgt = m.get<int>(s.p2p_cap);
    L.def_src = m.get<int>(s.def_cap);
    L.m2p_src = m.get<int>(s.m2p_cap);
    L.m2p_tgt = m.get<int>(s.m2p_cap);
    L.p2l_src = m.get<int>(s.p2l_cap);
    L.p2l_tgt = m.get<int>(s.p2l_cap);
    b.hash_keys = m.get<uint64_t>(kHashCap);
    b.tcount = m.get<unsigned long long>(5);
    b.totals = m.get<unsigned long long>(5);
    b.far = m.get<float4>(N);
    b.near = m.get<float4>(N);
    b.hflag = m.get<int>(kHashCap);
    b.hex = m.get<int>(kHashCap + 1);
    b.ukeys = m.get<uint64_t>(kHashCap);
    b.ukeys_alt = m.get<uint64_t>(kHashCap);
    b.uslot = m.get<uint32_t>(kHashCap);
    b.slot_class = m.get<int>(kHashCap);
    b.class_slot = m.get<int>(s.nclass_cap);
    b.tile_cells = m.get<int>((size_t)s.tile_cap * kTile);
    b.tile_key = m.get<uint64_t>(s.cell_cap);
    b.tile_key_alt = m.get<uint64_t>(s.cell_cap);
    b.tile_val = m.get<uint32_t>(s.cell_cap);
    b.tile_val_alt = m.get<uint32_t>(s.cell_cap);
    b.tile_hist = m.get<uint32_t>(radix_scratch_elems(s.cell_cap));
    b.bitmap = m.get<uint32_t>((size_t)s.tile_cap * s.nwords);
    b.tile_cnt = m.get<int>(s.tile_cap);
    b.entry_base = m.get<int>(s.tile_cap + 1);
    b.word_prefix = m.get<int>((size_t)s.tile_cap * s.nwords);
    b.entry_class = m.get<int>(s.nent_cap);
    b.src = m.get<int>((size_t)s.nent_cap * kTile);
    b.M = m.get<float>((size_t)cc * P2pad);
    b.Lx = m.get<float>((size_t)cc * P2pad);
    b.mtmp = m.get<float>((size_t)cc * P2pad);
    if (s.tensor) {
        b.units = m.get<M2LUnit>(s.units_cap);
        b.unit_base = m.get<int>(s.tile_cap + 1);
        b.tile_units = m.get<int>(s.units_cap);
        b.partial = m.get<float>((size_t)s.units_cap * 128 * P2pad);
    }

    // constant inputs: system offsets, selection table, operators and the class-key table
    cudaStream_t st = pl.st;
    {
        std::vector<int> off32(nsys + 1);
        for (int sy = 0; sy <= nsys; ++sy) off32[sy] = (int)offsets[sy];
        FMM_CUDA_TRY(cudaMemcpy(b.sys_off, off32.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice));
    }
    if (sel) {
        uint8_t *d = m.get<uint8_t>((size_t)kSelNB * kSelNB);
        FMM_CUDA_TRY(cudaMemcpy(d, sel, (size_t)kSelNB * kSelNB, cudaMemcpyHostToDevice));
        b.sel = d;
    }
    const size_t shift_n = (size_t)8 * P2pad * P2pad;
    float *m2m = m.get<float>(shift_n), *l2l = m.get<float>(shift_n);
    FMM_CUDA_TRY(cudaMemcpy(m2m, get<float>(ws, "m2m"), sizeof(float) * shift_n, cudaMemcpyDeviceToDevice));
    FMM_CUDA_TRY(cudaMemcpy(l2l, get<float>(ws, "l2l"), sizeof(float) * shift_n, cudaMemcpyDeviceToDevice));
    b.m2m = m2m;
    b.l2l = l2l;
    if (s.p >= kFp64TopP) {
        double *m64 = m.get<double>(shift_n), *l64 = m.get<double>(shift_n);
        FMM_CUDA_TRY(cudaMemcpy(m64, get<double>(ws, "m2m64"), sizeof(double) * shift_n, cudaMemcpyDeviceToDevice));
        FMM_CUDA_TRY(cudaMemcpy(l64, get<double>(ws, "l2l64"), sizeof(double) * shift_n, cudaMemcpyDeviceToDevice));
        b.m2m64 = m64;
        b.l2l64 = l64;
    }
    // every class operator built so far for this p, in the workspace's slots
    const int nops = std::max(ws.table_slots, 1);
    pl.operators = ws.table_slots;
    float *table = m.get<float>((size_t)nops * P2pad * P2pad);
    FMM_CUDA_TRY(cudaMemcpy(table, get<float>(ws, "table"), sizeof(float) * (size_t)ws.table_slots * P2pad * P2pad,
                            cudaMemcpyDeviceToDevice));
    b.table = table;
    if (s.tensor) {
        unsigned char *split = m.get<unsigned char>(m2l_split_bytes(P2pad, s.bf16, nops));
        launch_split_tables(s.bf16, table, 0, ws.table_slots, P2pad, split, st);
        b.tsplit = split;
    }
    {
        std::vector<uint64_t> hk(s.class_hcap, kHashEmpty);
        std::vector<int> hs(s.class_hcap, 0);
        for (const auto &kv : ws.class_cache) {
            uint32_t h = (uint32_t)((kv.first * 0x9e3779b97f4a7c15ull) >> 40) & (s.class_hcap - 1);
            while (hk[h] != kHashEmpty) h = (h + 1) & (s.class_hcap - 1);
            hk[h] = kv.first;
            hs[h] = kv.second;
        }
        uint64_t *dk = m.get<uint64_t>(s.class_hcap);
        int *ds = m.get<int>(s.class_hcap);
        FMM_CUDA_TRY(cudaMemcpy(dk, hk.data(), sizeof(uint64_t) * s.class_hcap, cudaMemcpyHostToDevice));
        FMM_CUDA_TRY(cudaMemcpy(ds, hs.data(), sizeof(int) * s.class_hcap, cudaMemcpyHostToDevice));
        b.chash_keys = dk;
        b.chash_slots = ds;
    }
    // kernel attributes are set outside the capture (the sizing solve may not
    // have run the hybrid kernels)
    const int rows_smem = (int)((size_t)32 * (P2pad + 1) * sizeof(float));
    if (rows_smem > 48 * 1024) {
        set_smem_limit_once((const void *)k_p2l, rows_smem);
    }
    if (s.hybrid && m2p_smem(s.p, P2pad) > 48 * 1024)
        set_smem_limit_once((const void *)k_m2p, (int)m2p_smem(s.p, P2pad));
    set_carveout_once((const void *)k_p2p, cudaSharedmemCarveoutMaxShared);
    FMM_CUDA_TRY(cudaStreamSynchronize(st));

    // capture
    const int64_t launches0 = g_launch_count;
    FMM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_plan(s, b, st, pl.fs, pl.tree, pl.fork, pl.join);
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    FMM_CUDA_TRY(cudaStreamEndCapture(st, &pl.graph));
    pl.graph_kernels = g_launch_count - launches0;
    size_t nodes = 0;
    FMM_CUDA_TRY(cudaGraphGetNodes(pl.graph, nullptr, &nodes));
    pl.graph_nodes = (int64_t)nodes;
    FMM_CUDA_TRY(cudaGraphInstantiate(&pl.exec, pl.graph, 0));
}

// One replay of a plan on `stream`: the inputs copied into the plan (unless they
// are its own buffers), one graph launch, the results copied out.
void plan_execute(fmm_plan &pl, const float *xyz, const float *q, float *phi, float *grad, cudaStream_t st)
{
    const size_t n = (size_t)pl.s.N;
    if (xyz && xyz != pl.xyz)
        FMM_CUDA_TRY(cudaMemcpyAsync(pl.xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st));
    if (q && q != pl.q) FMM_CUDA_TRY(cudaMemcpyAsync(pl.q, q, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaGraphLaunch(pl.exec, st));
    if (phi && phi != pl.phi)
        FMM_CUDA_TRY(cudaMemcpyAsync(phi, pl.phi, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    if (grad && grad != pl.grad)
        FMM_CUDA_TRY(cudaMemcpyAsync(grad, pl.grad, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st));
}

// One replay of a plan made with caller_arrays on the caller's arrays, in place:
// their addresses go to the plan's pointer block (one small copy ahead of the
// graph on `st`; the pinned source is rewritten only after the replay's check
// has waited for the stream).
void plan_execute_io(fmm_plan &pl, const float *xyz, const float *q, float *phi, float *grad, cudaStream_t st)
{
    pl.hio->xyz = xyz;
    pl.hio->q = q;
    pl.hio->phi = phi;
    pl.hio->grad = grad;
    FMM_CUDA_TRY(cudaMemcpyAsync(pl.io, pl.hio, sizeof(IoPtrs), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaGraphLaunch(pl.exec, st));
}

// Waits for `stream` and raises what the last replay's flags report.
void plan_check(fmm_plan &pl, cudaStream_t st)
{
    // both read-backs queued behind the replay, then one wait
    if (!pl.hcheck) FMM_CUDA_TRY(cudaMallocHost(&pl.hcheck, sizeof(int) * (kNumFlags + kSzWords)));
    FMM_CUDA_TRY(cudaMemcpyAsync(pl.hcheck, pl.b.flags, sizeof(int) * kNumFlags, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(pl.hcheck + kNumFlags, pl.b.sz, sizeof(int) * kSzWords, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    const int *f = pl.hcheck, *sz = pl.hcheck + kNumFlags;
    if (f[kFlagNonfinite]) throw Error{FMM_ERR_NONFINITE, "a coordinate is NaN or infinite"};
    if (f[kFlagTimeout]) throw Error{FMM_ERR_TIMEOUT, "a bounded device-side wait expired (M2L pipeline)"};
    if (sz[kSzAbort] || f[kFlagHashFull] || f[kFlagClassRange] || f[kFlagStack])
        throw Error{FMM_ERR_CAPACITY, "the replay exceeded a capacity of the plan or met an offset class it has "
                                      "no operator for; its results are invalid (create a new plan)"};
}

// A plan captured from the workspace's last solve (its sizes, operators and
// classes).  Its particle and result arrays are its own, or, for the plan that
// repeated calls replay (caller_arrays), the caller's of each replay: their
// addresses go to the plan's pointer block before each launch (plan_execute_io),
// so that any arrays are read and written in place.
fmm_plan *plan_from_last_solve(Workspace &ws, int64_t N, int nsys, const int64_t *off, int p, double theta,
                               int ncrit, const fmm_options &o, const uint8_t *sel, double headroom,
                               bool caller_arrays = false)
{
    std::unique_ptr<fmm_plan> pl(new fmm_plan());
    FMM_CUDA_TRY(cudaGetDevice(&pl->device));
    if (caller_arrays) {
        pl->io = pl->mem.get<IoPtrs>(1);
        FMM_CUDA_TRY(cudaMallocHost(reinterpret_cast<void **>(&pl->hio), sizeof(IoPtrs)));
    } else {
        pl->xyz = pl->mem.get<float>(3 * (size_t)N);
        pl->q = pl->mem.get<float>((size_t)N);
        pl->phi = pl->mem.get<float>((size_t)N);
        pl->grad = pl->mem.get<float>(3 * (size_t)N);
    }
    pl->s = plan_shape(ws, N, nsys, p, theta, ncrit, o, sel != nullptr, headroom);
    build_plan(*pl, ws, off, sel);
    return pl.release();
}

// The solve behind the public entry points (device arrays, the workspace
// locked).  With fmm_options.replay and no statistics: a call whose key (sizes,
// order, MAC, options, system offsets, selection table) equals the previous
// call's captures a plan after solving, and later calls with that key replay
// it -- one graph launch, every size on the device, the same arithmetic, so the
// same bits as a plain solve.  A replay that outgrows the plan's capacities (or
// meets an offset class it holds no operator for) is solved again plainly and
// the plan is dropped.
void solve_api(Workspace &ws, const float *xyz, const float *q, int64_t N, int nsys, const int64_t *off, int p,
               double theta, int ncrit, float *phi, float *grad, cudaStream_t stream, const fmm_options &o,
               fmm_stats *stats, const uint8_t *sel)
{
    if (!o.replay || stats || o.serialize_phases) {
        solve_locked(ws, xyz, q, N, nsys, off, p, theta, ncrit, phi, grad, stream, o, stats, sel);
        return;
    }
    Workspace::ReplayKey key;
    key.N = N;
    key.nsys = nsys;
    key.p = p;
    key.ncrit = ncrit;
    key.max_depth = o.max_depth;
    key.precision = o.precision_mode;
    key.select_mode = o.select_mode;
    key.unit_blocks = o.m2l_unit_blocks;
    key.theta = theta;
    key.off.assign(off, off + nsys + 1);
    if (sel) key.sel.assign(sel, sel + (size_t)kSelNB * kSelNB);
    if (ws.replay_plan && ws.replay_key == key) {
        try {
            plan_execute_io(*ws.replay_plan, xyz, q, phi, grad, stream);
            plan_check(*ws.replay_plan, stream);
            // (calls that alternate between keys then solve the other keys plainly
            // instead of capturing a plan at every other call)
            ws.last_key = std::move(key);
            ws.have_last = true;
            return;
        } catch (const Error &e) {
            if (e.code != FMM_ERR_CAPACITY) throw;
        }
        delete ws.replay_plan;  // outgrown: solve plainly below
        ws.replay_plan = nullptr;
    }
    solve_locked(ws, xyz, q, N, nsys, off, p, theta, ncrit, phi, grad, stream, o, nullptr, sel);
    if (ws.have_last && ws.last_key == key && !(ws.replay_plan && ws.replay_key == key)) {
        delete ws.replay_plan;
        ws.replay_plan = nullptr;
        try {
            ws.replay_plan = plan_from_last_solve(ws, N, nsys, off, p, theta, ncrit, o, sel, 1.25, true);
            ws.replay_key = key;
        } catch (const Error &) {
            // no plan for this key (the solve itself succeeded): later calls solve plainly
            cudaGetLastError();
        }
    }
    ws.last_key = std::move(key);
    ws.have_last = true;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" {

void fmm_default_options(fmm_options *opt)
{
    if (!opt) return;
    opt->max_depth = 0;
    opt->precision_mode = FMM_PREC_FP32;
    opt->select_mode = FMM_SELECT_PLAIN;
    opt->deterministic = 1;
    opt->select_table = nullptr;
    opt->m2l_unit_blocks = 0;
    opt->serialize_phases = 0;
    opt->replay = 1;
}

fmm_status fmm_laplace3d_ex(const float *xyz, const float *q, int64_t N, int p, double theta,
                            int ncrit, float *phi, float *grad, void *stream,
                            const fmm_options *opt, fmm_stats *stats)
{
    return guarded([&] {
        const fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, ncrit, phi, grad, o);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        const int64_t off[2] = {0, N};
        solve_api(ws, xyz, q, N, 1, off, p, theta, ncrit, phi, grad, (cudaStream_t)stream, o, stats, sel);
    });
}

fmm_status fmm_laplace3d(const float *xyz, const float *q, int64_t N, int p, double theta,
                         int ncrit, float *phi, float *grad, void *stream)
{
    return fmm_laplace3d_ex(xyz, q, N, p, theta, ncrit, phi, grad, stream, nullptr, nullptr);
}

fmm_status fmm_laplace3d_host(const float *xyz_host, const float *q_host, int64_t N, int p,
                              double theta, int ncrit, float *phi_host, float *grad_host,
                              void *stream, const fmm_options *opt, fmm_stats *stats)
{
    return guarded([&] {
        const fmm_options o = resolve_opts(opt);
        validate(xyz_host, q_host, N, p, theta, ncrit, phi_host, grad_host, o);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        cudaStream_t st = (cudaStream_t)stream;
        float *xd = need<float>(ws, "host_xyz", 3 * (size_t)N, st);
        float *qd = need<float>(ws, "host_q", (size_t)N, st);
        float *pd = need<float>(ws, "host_phi", (size_t)N, st);
        float *gd = need<float>(ws, "host_grad", 3 * (size_t)N, st);
        FMM_CUDA_TRY(cudaMemcpyAsync(xd, xyz_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(qd, q_host, sizeof(float) * N, cudaMemcpyHostToDevice, st));
        const int64_t off[2] = {0, N};
        solve_api(ws, xd, qd, N, 1, off, p, theta, ncrit, pd, gd, st, o, stats, sel);
        FMM_CUDA_TRY(cudaMemcpyAsync(phi_host, pd, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(grad_host, gd, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

fmm_status fmm_laplace3d_batched(const float *xyz, const float *q, const int64_t *offsets,
                                 int nsys, int p, double theta, int ncrit, float *phi, float *grad,
                                 void *stream, const fmm_options *opt, fmm_stats *stats)
{
    return guarded([&] {
        if (!offsets || nsys < 1) throw Error{FMM_ERR_ARG, "offsets must hold nsys + 1 >= 2 entries"};
        if (offsets[0] != 0) throw Error{FMM_ERR_ARG, "offsets[0] must be 0"};
        for (int sy = 0; sy < nsys; ++sy)
            if (offsets[sy + 1] <= offsets[sy]) throw Error{FMM_ERR_ARG, "every system needs at least one particle"};
        const int64_t N = offsets[nsys];
        const fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, ncrit, phi, grad, o);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        solve_api(ws, xyz, q, N, nsys, offsets, p, theta, ncrit, phi, grad, (cudaStream_t)stream, o,
                     stats, sel);
    });
}

// ---------------------------------------------------------------- hybrid selection

fmm_status fmm_selection_table(int select_mode, int p, double theta, int precision_mode,
                               unsigned char *table)
{
    return guarded([&] {
        if (!table) throw Error{FMM_ERR_ARG, "null table"};
        if (p < 1 || p > 20 || !(theta > 0.0 && theta < 1.0)) throw Error{FMM_ERR_ARG, "p or theta out of range"};
        if (precision_mode < FMM_PREC_FP32 || precision_mode > FMM_PREC_BF16X3)
            throw Error{FMM_ERR_ARG, "precision_mode must be FMM_PREC_*"};
        if (select_mode != FMM_SELECT_AUTOTUNE && select_mode != FMM_SELECT_LEARNED)
            throw Error{FMM_ERR_ARG, "select_mode must be FMM_SELECT_AUTOTUNE or FMM_SELECT_LEARNED"};
        fmm_options o;
        fmm_default_options(&o);
        o.select_mode = select_mode;
        o.precision_mode = precision_mode;
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        std::memcpy(table, selection_table(ws, o, p, theta), (size_t)kSelNB * kSelNB);
    });
}

fmm_status fmm_tune_ncrit(const float *xyz, const float *q, int64_t N, int p, double theta, void *stream,
                          const fmm_options *opt, const int *candidates, int ncand, float *ms, int *best)
{
    return guarded([&] {
        if (!candidates || ncand < 1 || !best) throw Error{FMM_ERR_ARG, "need candidates, ncand >= 1 and best"};
        for (int k = 0; k < ncand; ++k)
            if (candidates[k] < 1) throw Error{FMM_ERR_ARG, "every candidate ncrit must be >= 1"};
        const fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, 1, xyz, xyz, o);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        cudaStream_t st = (cudaStream_t)stream;
        float *phi = need<float>(ws, "tune_phi", (size_t)N, st);
        float *grad = need<float>(ws, "tune_grad", 3 * (size_t)N, st);
        const int64_t off[2] = {0, N};
        float best_ms = 1e30f;
        for (int k = 0; k < ncand; ++k) {
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                fmm_stats s{};
                solve_locked(ws, xyz, q, N, 1, off, p, theta, candidates[k], phi, grad, st, o, &s, sel);
                if (rep > 0) t = std::min(t, s.ms_total);  // the first solve sizes the buffers
            }
            if (ms) ms[k] = t;
            if (t < best_ms) {
                best_ms = t;
                *best = candidates[k];
            }
        }
        ws.have_solve = false;
    });
}

fmm_status fmm_tune_schedule(const float *xyz, const float *q, int64_t N, const int64_t *offsets, int nsys,
                             int p, double theta, void *stream, const fmm_options *opt, const int *ncrit_cand,
                             int nncrit, const int *unit_cand, int nunit, float *ms, int *best_ncrit,
                             int *best_unit)
{
    return guarded([&] {
        if (!ncrit_cand || nncrit < 1 || !unit_cand || nunit < 1 || !best_ncrit || !best_unit)
            throw Error{FMM_ERR_ARG, "need candidate lists and result pointers"};
        for (int k = 0; k < nncrit; ++k)
            if (ncrit_cand[k] < 1) throw Error{FMM_ERR_ARG, "every candidate ncrit must be >= 1"};
        for (int u = 0; u < nunit; ++u)
            if (unit_cand[u] < 0) throw Error{FMM_ERR_ARG, "unit candidates must be >= 0"};
        std::vector<int64_t> off1 = {0, N};
        const int64_t *off = offsets ? offsets : off1.data();
        if (!offsets) nsys = 1;
        if (nsys < 1 || off[0] != 0) throw Error{FMM_ERR_ARG, "offsets must start at 0"};
        for (int sy = 0; sy < nsys; ++sy)
            if (off[sy + 1] <= off[sy]) throw Error{FMM_ERR_ARG, "every system needs at least one particle"};
        N = off[nsys];
        fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, 1, xyz, xyz, o);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        cudaStream_t st = (cudaStream_t)stream;
        float *phi = need<float>(ws, "tune_phi", (size_t)N, st);
        float *grad = need<float>(ws, "tune_grad", 3 * (size_t)N, st);
        float best_ms = 1e30f;
        for (int k = 0; k < nncrit; ++k)
            for (int u = 0; u < nunit; ++u) {
                o.m2l_unit_blocks = unit_cand[u];
                float t = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    fmm_stats s{};
                    solve_locked(ws, xyz, q, N, nsys, off, p, theta, ncrit_cand[k], phi, grad, st, o, &s, sel);
                    if (rep > 0) t = std::min(t, s.ms_total);  // the first solve sizes the buffers
                }
                if (ms) ms[k * nunit + u] = t;
                if (t < best_ms) {
                    best_ms = t;
                    *best_ncrit = ncrit_cand[k];
                    *best_unit = unit_cand[u];
                }
            }
        ws.have_solve = false;
    });
}

fmm_status fmm_cost_model_train(int precision_mode, int p_lo, int p_hi, int steps, uint64_t seed,
                                fmm_cost_model_info *info)
{
    return guarded([&] {
        if (p_lo < 1 || p_hi > 20 || p_lo > p_hi) throw Error{FMM_ERR_ARG, "need 1 <= p_lo <= p_hi <= 20"};
        if (steps < 1) throw Error{FMM_ERR_ARG, "steps must be >= 1"};
        if (precision_mode < FMM_PREC_FP32 || precision_mode > FMM_PREC_BF16X3)
            throw Error{FMM_ERR_ARG, "precision_mode must be FMM_PREC_*"};
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        ensure_streams(ws);
        cudaStream_t st = ws.main_stream;
        cudaEvent_t e0, e1, e2;
        FMM_CUDA_TRY(cudaEventCreate(&e0));
        FMM_CUDA_TRY(cudaEventCreate(&e1));
        FMM_CUDA_TRY(cudaEventCreate(&e2));
        FMM_CUDA_TRY(cudaEventRecord(e0, st));
        // samples: P2P times on artificial leaves (cost independent of sep and p, which
        // are drawn at random), M2L times from artificial solves at each (p, theta)
        SplitMix64 rng{seed};
        Samples s;
        auto add = [&](double lnt, double lns, double sep, double pp, double t0, double t1, float m0, float m1) {
            s.x.insert(s.x.end(), {(float)lnt, (float)lns, (float)sep, (float)pp});
            s.t.insert(s.t.end(), {(float)t0, (float)t1});
            s.m.insert(s.m.end(), {m0, m1});
        };
        int64_t np2p = 0, nm2l = 0;
        for (const P2PTiming &g : p2p_timings(ws)) {
            for (int r = 0; r < 2; ++r) {
                add(std::log2((double)g.nt), std::log2((double)g.ns), 1.4 + 2.4 * rng.uniform(),
                    p_lo + (p_hi - p_lo) * rng.uniform(), std::log(g.ns_per_pair), 0.0, 1.f, 0.f);
                ++np2p;
            }
        }
        const double thetas[4] = {0.35, 0.45, 0.55, 0.65};
        for (int pp = p_lo; pp <= p_hi; ++pp) {
            for (double th : thetas) {
                const double lt = std::log(m2l_ns_per_pair(ws, pp, th, precision_mode));
                for (int r = 0; r < 8; ++r) {
                    add(10.0 * rng.uniform(), 10.0 * rng.uniform(), 1.0 / th, pp, 0.0, lt, 0.f, 1.f);
                    ++nm2l;
                }
            }
        }
        FMM_CUDA_TRY(cudaEventRecord(e1, st));
        const std::vector<float> w0 = model_init(s, seed ^ 0xa5a5a5a5ull);
        model_set(ws.cm, w0.data(), st);
        float l0 = 0.f, l1 = 0.f;
        model_train(ws.cm, s, steps, 3e-3f, l0, l1, st);
        FMM_CUDA_TRY(cudaEventRecord(e2, st));
        FMM_CUDA_TRY(cudaEventSynchronize(e2));
        ws.cm.trained = true;
        ws.cm.last = s;
        for (auto it = ws.tables.begin(); it != ws.tables.end();)
            it = std::get<0>(it->first) == FMM_SELECT_LEARNED ? ws.tables.erase(it) : std::next(it);
        // the judge: agreement of the learned table with the pre-timed one over
        // counts up to 4096 (buckets < 43), worst case over the training grid
        float agree = 1.f;
        for (int pp = p_lo; pp <= p_hi; ++pp) {
            for (double th : thetas) {
                const std::vector<uint8_t> &a = pretimed_table(ws, pp, th, precision_mode);
                const std::vector<uint8_t> &b = learned_table(ws, pp, th);
                int same = 0, tot = 0;
                for (int i = 0; i < 43; ++i)
                    for (int j = 0; j < 43; ++j, ++tot) same += a[i * kSelNB + j] == b[i * kSelNB + j];
                agree = std::min(agree, (float)same / (float)tot);
            }
        }
        if (info) {
            info->n_samples_p2p = np2p;
            info->n_samples_m2l = nm2l;
            info->steps = steps;
            info->loss_initial = l0;
            info->loss_final = l1;
            info->agreement = agree;
            FMM_CUDA_TRY(cudaEventElapsedTime(&info->ms_pretime, e0, e1));
            FMM_CUDA_TRY(cudaEventElapsedTime(&info->ms_train, e1, e2));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
    });
}

fmm_status fmm_cost_model_get(float *params, int64_t n, int master)
{
    return guarded([&] {
        if (!params || n < FMM_COST_MODEL_PARAMS) throw Error{FMM_ERR_ARG, "params needs FMM_COST_MODEL_PARAMS floats"};
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.cm.w16) throw Error{FMM_ERR_ARG, "no cost model has been trained or set"};
        if (master) {
            FMM_CUDA_TRY(cudaMemcpy(params, ws.cm.w32, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
        } else {
            std::vector<__half> h(kMlpParams);
            FMM_CUDA_TRY(cudaMemcpy(h.data(), ws.cm.w16, sizeof(__half) * kMlpParams, cudaMemcpyDeviceToHost));
            for (int i = 0; i < kMlpParams; ++i) params[i] = __half2float(h[i]);
        }
    });
}

fmm_status fmm_cost_model_set(const float *params, int64_t n)
{
    return guarded([&] {
        if (!params || n != FMM_COST_MODEL_PARAMS) throw Error{FMM_ERR_ARG, "params must hold FMM_COST_MODEL_PARAMS floats"};
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(params[i])) throw Error{FMM_ERR_NONFINITE, "non-finite parameter"};
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        ensure_streams(ws);
        model_set(ws.cm, params, ws.main_stream);
        ws.cm.trained = true;
        for (auto it = ws.tables.begin(); it != ws.tables.end();)
            it = std::get<0>(it->first) == FMM_SELECT_LEARNED ? ws.tables.erase(it) : std::next(it);
    });
}

fmm_status fmm_cost_model_grad(const float *x, const float *t, const float *m, int64_t B, float *loss,
                               float *grad)
{
    return guarded([&] {
        if (!t || !m || !loss || !grad) throw Error{FMM_ERR_ARG, "null argument"};
        const Samples s = host_samples(x, t, m, B);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.cm.w16) throw Error{FMM_ERR_ARG, "no cost model has been trained or set"};
        ensure_streams(ws);
        model_grad(ws.cm, s, loss, grad, ws.main_stream);
    });
}

fmm_status fmm_cost_model_adam_step(const float *x, const float *t, const float *m, int64_t B, float lr,
                                    float *loss)
{
    return guarded([&] {
        if (!t || !m || !loss || !(lr > 0.f)) throw Error{FMM_ERR_ARG, "bad argument"};
        const Samples s = host_samples(x, t, m, B);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.cm.w16) throw Error{FMM_ERR_ARG, "no cost model has been trained or set"};
        ensure_streams(ws);
        model_adam_step(ws.cm, s, lr, loss, ws.main_stream);
        for (auto it = ws.tables.begin(); it != ws.tables.end();)
            it = std::get<0>(it->first) == FMM_SELECT_LEARNED ? ws.tables.erase(it) : std::next(it);
    });
}

fmm_status fmm_cost_model_predict(const float *x, int64_t B, float *y)
{
    return guarded([&] {
        if (!y) throw Error{FMM_ERR_ARG, "null y"};
        const Samples s = host_samples(x, nullptr, nullptr, B);
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.cm.w16) throw Error{FMM_ERR_ARG, "no cost model has been trained or set"};
        ensure_streams(ws);
        model_predict(ws.cm, s.x.data(), B, y, ws.main_stream);
    });
}

fmm_status fmm_cost_model_samples(float *x, float *t, float *m, int64_t capacity, int64_t *n)
{
    return guarded([&] {
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const int64_t k = ws.cm.last.size();
        if (n) *n = k;
        if (!x && !t && !m) return;
        if (!x || !t || !m || capacity < k) throw Error{FMM_ERR_ARG, "buffers too small"};
        std::memcpy(x, ws.cm.last.x.data(), sizeof(float) * 4 * k);
        std::memcpy(t, ws.cm.last.t.data(), sizeof(float) * 2 * k);
        std::memcpy(m, ws.cm.last.m.data(), sizeof(float) * 2 * k);
    });
}

fmm_status fmm_selftest_wait_timeout(int64_t polls, void *stream)
{
    return guarded([&] {
        if (polls < 1 || polls > (int64_t(1) << 26)) throw Error{FMM_ERR_ARG, "polls must be in [1, 2^26]"};
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        cudaStream_t st = (cudaStream_t)stream;
        int *flags = need<int>(ws, "selftest_flags", kNumFlags, st);
        FMM_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * kNumFlags, st));
        launch_wait_selftest((uint32_t)polls, flags, st);
        sync_point(ws, st, flags, {}, nullptr);  // raises FMM_ERR_TIMEOUT from the flag
    });
}

fmm_status fmm_direct(const float *xyz, const float *q, int64_t N, float *phi, float *grad,
                      void *stream)
{
    return guarded([&] {
        if (!xyz || !q || !phi || !grad) throw Error{FMM_ERR_ARG, "null pointer argument"};
        if (N < 1 || N >= (int64_t(1) << 31)) throw Error{FMM_ERR_ARG, "N must be in [1, 2^31)"};
        cudaStream_t st = (cudaStream_t)stream;
        k_direct<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(xyz, q, N, phi, grad);
        FMM_LAUNCH_CHECK();
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

fmm_status fmm_export(int what, void *dst, int64_t capacity, int64_t *needed)
{
    return guarded([&] {
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.have_solve) throw Error{FMM_ERR_ARG, "no solve has completed on this device"};
        int64_t bytes = 0;
        switch (what) {
            case FMM_EXPORT_BOX: bytes = 4 * sizeof(double) * ws.nsys; break;
            case FMM_EXPORT_KEYS: bytes = ws.N * sizeof(uint64_t); break;
            case FMM_EXPORT_ORDER: bytes = ws.N * sizeof(int32_t); break;
            case FMM_EXPORT_CELLS: bytes = (int64_t)ws.ncells * 6 * sizeof(int64_t); break;
            case FMM_EXPORT_P2P: bytes = ws.np2p * 2 * sizeof(int32_t); break;
            case FMM_EXPORT_M2L: bytes = ws.nm2l * 3 * sizeof(int32_t); break;
            case FMM_EXPORT_MULTIPOLE:
            case FMM_EXPORT_LOCAL: bytes = (int64_t)ws.ncells * ws.P2pad * sizeof(float); break;
            case FMM_EXPORT_SELECT: bytes = (int64_t)ws.sel_host.size(); break;
            case FMM_EXPORT_M2P: bytes = ws.nm2p * 2 * sizeof(int32_t); break;
            case FMM_EXPORT_P2L: bytes = ws.np2l * 2 * sizeof(int32_t); break;
            default: throw Error{FMM_ERR_ARG, "unknown export kind"};
        }
        if (needed) *needed = bytes;
        if (!dst) return;
        if (capacity < bytes) throw Error{FMM_ERR_ARG, "export buffer too small"};
        auto d2h = [](void *h, const void *d, size_t n) {
            if (n) FMM_CUDA_TRY(cudaMemcpy(h, d, n, cudaMemcpyDeviceToHost));
        };
        switch (what) {
            case FMM_EXPORT_BOX: d2h(dst, get<double>(ws, "box"), bytes); break;
            case FMM_EXPORT_KEYS: d2h(dst, get<uint64_t>(ws, "keys"), bytes); break;
            case FMM_EXPORT_ORDER: d2h(dst, get<uint32_t>(ws, "idx"), bytes); break;
            case FMM_EXPORT_MULTIPOLE: d2h(dst, get<float>(ws, "M"), bytes); break;
            case FMM_EXPORT_LOCAL: d2h(dst, get<float>(ws, "L"), bytes); break;
            case FMM_EXPORT_SELECT: std::memcpy(dst, ws.sel_host.data(), bytes); break;
            case FMM_EXPORT_CELLS: {
                const int n = ws.ncells;
                std::vector<int> lv(n), b(n), e(n), par(n), nch(n);
                std::vector<uint64_t> pre(n);
                d2h(lv.data(), get<int>(ws, "c_level"), n * sizeof(int));
                d2h(pre.data(), get<uint64_t>(ws, "c_prefix"), n * sizeof(uint64_t));
                d2h(b.data(), get<int>(ws, "c_begin"), n * sizeof(int));
                d2h(e.data(), get<int>(ws, "c_end"), n * sizeof(int));
                d2h(par.data(), get<int>(ws, "c_parent"), n * sizeof(int));
                d2h(nch.data(), get<int>(ws, "c_nchild"), n * sizeof(int));
                int64_t *o = static_cast<int64_t *>(dst);
                for (int i = 0; i < n; ++i) {
                    o[6 * i] = lv[i];
                    o[6 * i + 1] = (int64_t)pre[i];
                    o[6 * i + 2] = b[i];
                    o[6 * i + 3] = e[i];
                    o[6 * i + 4] = par[i];
                    o[6 * i + 5] = nch[i];
                }
                break;
            }
            case FMM_EXPORT_P2P: {
                const int64_t n = ws.np2p;
                std::vector<int> t(n), s(n);
                d2h(t.data(), get<int>(ws, "p2p_tgt"), n * sizeof(int));
                d2h(s.data(), get<int>(ws, "p2p_src"), n * sizeof(int));
                int32_t *o = static_cast<int32_t *>(dst);
                for (int64_t i = 0; i < n; ++i) {
                    o[2 * i] = t[i];
                    o[2 * i + 1] = s[i];
                }
                break;
            }
            case FMM_EXPORT_M2P:
            case FMM_EXPORT_P2L: {
                const bool m2p = what == FMM_EXPORT_M2P;
                const int64_t n = m2p ? ws.nm2p : ws.np2l;
                std::vector<int> t(n), s(n);
                d2h(t.data(), get<int>(ws, m2p ? "m2p_tgt" : "p2l_tgt"), n * sizeof(int));
                d2h(s.data(), get<int>(ws, m2p ? "m2p_src" : "p2l_src"), n * sizeof(int));
                int32_t *o = static_cast<int32_t *>(dst);
                for (int64_t i = 0; i < n; ++i) {
                    o[2 * i] = t[i];
                    o[2 * i + 1] = s[i];
                }
                break;
            }
            case FMM_EXPORT_M2L: {
                const int64_t n = ws.nm2l;
                std::vector<int> t(n), s(n), k(n);
                d2h(t.data(), get<int>(ws, "m2l_tgt"), n * sizeof(int));
                d2h(s.data(), get<int>(ws, "m2l_src"), n * sizeof(int));
                d2h(k.data(), get<uint32_t>(ws, "m2l_slot"), n * sizeof(int));
                int32_t *o = static_cast<int32_t *>(dst);
                for (int64_t i = 0; i < n; ++i) {
                    o[3 * i] = t[i];
                    o[3 * i + 1] = s[i];
                    o[3 * i + 2] = k[i];
                }
                break;
            }
        }
    });
}

fmm_status fmm_cost_model_pick_ncrit(const float *xyz, const float *q, int64_t N, int p, double theta, void *stream,
                                     const fmm_options *opt, const int *candidates, int ncand, float *pred_ms,
                                     int *best)
{
    return guarded([&] {
        if (!candidates || ncand < 1 || !best) throw Error{FMM_ERR_ARG, "need candidates and best"};
        const fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, 1, xyz, xyz, o);
        for (int k = 0; k < ncand; ++k)
            if (candidates[k] < 1) throw Error{FMM_ERR_ARG, "ncrit candidates must be >= 1"};
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        if (!ws.cm.trained) throw Error{FMM_ERR_ARG, "no cost model: train or set one first"};
        ensure_streams(ws);
        cudaStream_t cs = (cudaStream_t)stream, st = ws.main_stream;
        const uint8_t *sel = selection_table(ws, o, p, theta);
        const SolveCal cal = solve_calibration(ws, p, theta, o.precision_mode);
        const int64_t off[2] = {0, N};
        unsigned long long *hist = need<unsigned long long>(ws, "pick_hist", (size_t)kSelNB * kSelNB, st);
        double *cost = need<double>(ws, "pick_cost", 2, st);
        // the network's P2P prediction is scaled to the P2P kernel's measured time
        // on the calibration solves (the network gives how the time varies with
        // the leaf sizes; the solves fix its scale in a real solve)
        double net_cal = 0.0, meas_cal = 0.0;
        for (int k = 0; k < 2; ++k) {
            FMM_CUDA_TRY(cudaMemcpyAsync(hist, cal.hist[k].data(), sizeof(unsigned long long) * kSelNB * kSelNB,
                                         cudaMemcpyHostToDevice, st));
            k_mlp_solve_cost<<<1, 256, 0, st>>>(ws.cm.w16, (float)p, (float)(1.0 / theta), hist, 0ull, cost);
            FMM_LAUNCH_CHECK();
            double h[2];
            FMM_CUDA_TRY(cudaMemcpyAsync(h, cost, sizeof(h), cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            net_cal += h[0];
            meas_cal += cal.p2p_ns[k];
        }
        const double p2p_scale = net_cal > 0.0 ? meas_cal / net_cal : 1.0;
        double best_ns = 1e300;
        for (int k = 0; k < ncand; ++k) {
            // the candidate's tree and interaction lists (no evaluation), then the
            // network over them
            solve_locked(ws, xyz, q, N, 1, off, p, theta, candidates[k], nullptr, nullptr, cs, o, nullptr, sel, false,
                         true);
            const int64_t np2p = ws.shape.tot[1], nm2l = ws.shape.tot[0];
            FMM_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kSelNB * kSelNB, st));
            if (np2p > 0) {
                k_pair_bucket_hist<<<grid_for(np2p, 256), 256, 0, st>>>(get<int>(ws, "p2p_tgt"), get<int>(ws, "p2p_src"),
                                                                      np2p, get<int>(ws, "c_begin"),
                                                                      get<int>(ws, "c_end"), hist);
                FMM_LAUNCH_CHECK();
            }
            k_mlp_solve_cost<<<1, 256, 0, st>>>(ws.cm.w16, (float)p, (float)(1.0 / theta), hist,
                                               (unsigned long long)nm2l, cost);
            FMM_LAUNCH_CHECK();
            double h[2];
            FMM_CUDA_TRY(cudaMemcpyAsync(h, cost, sizeof(h), cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            // the network's P2P time (scaled), the calibrated M2L and per-cell times
            const double ns = p2p_scale * h[0] + cal.ns_block * (double)ws.shape.nent +
                              cal.ns_cell * (double)ws.shape.ncells + cal.ns_fixed;
            if (pred_ms) pred_ms[k] = (float)(ns * 1e-6);
            if (ns < best_ns) {
                best_ns = ns;
                *best = candidates[k];
            }
        }
        ws.have_solve = false;  // the workspace holds lists, not a finished solve
    });
}

fmm_status fmm_measure_fp32(double *ffma_tflops, double *body_inter_per_s, void *stream)
{
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        int dev = 0, nsm = 152;
        FMM_CUDA_TRY(cudaGetDevice(&dev));
        FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const int ffma_blocks = nsm * 8, body_blocks = nsm * kP2PBlocksPerSM;
        float *out = need<float>(ws, "measure_out", (size_t)std::max(ffma_blocks * 256, body_blocks * 128), st);
        cudaEvent_t e0, e1;
        FMM_CUDA_TRY(cudaEventCreate(&e0));
        FMM_CUDA_TRY(cudaEventCreate(&e1));
        auto timed = [&](auto launch) {
            launch(true);  // warm-up
            FMM_CUDA_TRY(cudaEventRecord(e0, st));
            launch(false);
            FMM_CUDA_TRY(cudaEventRecord(e1, st));
            FMM_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            FMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            return (double)ms;
        };
        const int iters = 20000, reps = 4000;
        const double ms_ffma = timed([&](bool warm) {
            k_ffma_stream<<<ffma_blocks, 256, 0, st>>>(out, warm ? 100 : iters, 1.0001f);
            FMM_LAUNCH_CHECK();
        });
        const double ms_body = timed([&](bool warm) {
            k_p2p_body<<<body_blocks, 128, 0, st>>>(out, warm ? 10 : reps);
            FMM_LAUNCH_CHECK();
        });
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (ffma_tflops) *ffma_tflops = (double)ffma_blocks * 256 * iters * 16 * 2 / (ms_ffma * 1e-3) / 1e12;
        if (body_inter_per_s) *body_inter_per_s = (double)body_blocks * 128 * reps * 32 / (ms_body * 1e-3);
    });
}

// ---------------------------------------------------------------- captured plans

fmm_status fmm_plan_create(fmm_plan **plan, const float *xyz, const float *q, int64_t N, const int64_t *offsets,
                           int nsys, int p, double theta, int ncrit, const fmm_options *opt, double headroom,
                           void *stream)
{
    return guarded([&] {
        if (!plan) throw Error{FMM_ERR_ARG, "null plan pointer"};
        *plan = nullptr;
        if (headroom == 0.0) headroom = 1.25;
        if (!(headroom >= 1.0 && headroom <= 16.0)) throw Error{FMM_ERR_ARG, "headroom must be in [1, 16]"};
        std::vector<int64_t> off;
        if (offsets) {
            if (nsys < 1) throw Error{FMM_ERR_ARG, "offsets must hold nsys + 1 >= 2 entries"};
            if (offsets[0] != 0) throw Error{FMM_ERR_ARG, "offsets[0] must be 0"};
            for (int sy = 0; sy < nsys; ++sy)
                if (offsets[sy + 1] <= offsets[sy]) throw Error{FMM_ERR_ARG, "every system needs at least one particle"};
            if (offsets[nsys] != N) throw Error{FMM_ERR_ARG, "offsets[nsys] must equal N"};
            off.assign(offsets, offsets + nsys + 1);
        } else {
            if (nsys != 1) throw Error{FMM_ERR_ARG, "without offsets nsys must be 1"};
            off = {0, N};
        }
        const fmm_options o = resolve_opts(opt);
        validate(xyz, q, N, p, theta, ncrit, xyz, xyz, o);
        std::unique_ptr<fmm_plan> pl(new fmm_plan());
        FMM_CUDA_TRY(cudaGetDevice(&pl->device));
        pl->xyz = pl->mem.get<float>(3 * (size_t)N);
        pl->q = pl->mem.get<float>((size_t)N);
        pl->phi = pl->mem.get<float>((size_t)N);
        pl->grad = pl->mem.get<float>(3 * (size_t)N);
        cudaStream_t cs = (cudaStream_t)stream;
        FMM_CUDA_TRY(cudaMemcpyAsync(pl->xyz, xyz, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, cs));
        FMM_CUDA_TRY(cudaMemcpyAsync(pl->q, q, sizeof(float) * N, cudaMemcpyDeviceToDevice, cs));
        Workspace &ws = workspace_for_current_device();
        std::lock_guard<std::mutex> lk(ws.mu);
        const uint8_t *sel = selection_table(ws, o, p, theta);
        // the sizing solve (it also builds the operators of its classes)
        solve_locked(ws, pl->xyz, pl->q, N, nsys, off.data(), p, theta, ncrit, pl->phi, pl->grad, cs, o, nullptr, sel);
        FMM_CUDA_TRY(cudaStreamSynchronize(cs));
        pl->s = plan_shape(ws, N, nsys, p, theta, ncrit, o, sel != nullptr, headroom);
        build_plan(*pl, ws, off.data(), sel);
        *plan = pl.release();
    });
}

fmm_status fmm_plan_execute(fmm_plan *plan, const float *xyz, const float *q, float *phi, float *grad, void *stream)
{
    return guarded([&] {
        if (!plan) throw Error{FMM_ERR_ARG, "null plan"};
        int dev = 0;
        FMM_CUDA_TRY(cudaGetDevice(&dev));
        if (dev != plan->device) throw Error{FMM_ERR_ARG, "the plan belongs to another device"};
        plan_execute(*plan, xyz, q, phi, grad, (cudaStream_t)stream);
    });
}

fmm_status fmm_plan_check(fmm_plan *plan, void *stream)
{
    return guarded([&] {
        if (!plan) throw Error{FMM_ERR_ARG, "null plan"};
        plan_check(*plan, (cudaStream_t)stream);
    });
}

fmm_status fmm_plan_buffers(fmm_plan *plan, float **xyz, float **q, float **phi, float **grad)
{
    return guarded([&] {
        if (!plan) throw Error{FMM_ERR_ARG, "null plan"};
        if (xyz) *xyz = plan->xyz;
        if (q) *q = plan->q;
        if (phi) *phi = plan->phi;
        if (grad) *grad = plan->grad;
    });
}

fmm_status fmm_plan_info(fmm_plan *plan, fmm_plan_info_t *info)
{
    return guarded([&] {
        if (!plan || !info) throw Error{FMM_ERR_ARG, "null argument"};
        const PlanShape &s = plan->s;
        int sz[kSzWords];
        FMM_CUDA_TRY(cudaDeviceSynchronize());
        FMM_CUDA_TRY(cudaMemcpy(sz, plan->b.sz, sizeof(sz), cudaMemcpyDeviceToHost));
        *info = fmm_plan_info_t{};
        info->N = s.N;
        info->nsys = s.nsys;
        info->levels = s.levels;
        info->cell_cap = s.cell_cap;
        info->tile_cap = s.tile_cap;
        info->class_cap = s.nclass_cap;
        info->entry_cap = s.nent_cap;
        info->unit_cap = s.units_cap;
        info->m2l_cap = s.m2l_cap;
        info->p2p_cap = s.p2p_cap;
        info->operators = plan->operators;
        info->graph_nodes = plan->graph_nodes;
        info->graph_kernels = plan->graph_kernels;
        info->last_cells = sz[kSzCells];
        info->last_leaves = sz[kSzLeaves];
        info->last_classes = sz[kSzClasses];
        info->last_entries = sz[kSzEntries];
        info->last_units = sz[kSzUnits];
        info->last_valid = sz[kSzAbort] == 0;
    });
}

void fmm_plan_destroy(fmm_plan *plan) { delete plan; }

const char *fmm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
