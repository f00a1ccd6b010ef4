// kernels.cuh -- kernel declarations and the device-side data layout shared by
// the translation units of the CUDA path.
#pragma once

#include <cuda_fp16.h>

#include <climits>

#include <vector>

#include "common.cuh"

namespace fmm {

// Device error flags (int[kNumFlags]).
enum {
    kFlagNonfinite = 0,   // NaN/Inf coordinate
    kFlagHashFull = 1,    // offset-class hash table full
    kFlagClassRange = 2,  // an offset component does not fit the class key
    kFlagStack = 3,       // traversal stack overflow
    kFlagTimeout = 4,     // a bounded device-side wait expired
    kNumFlags = 8
};

// Device-side sizes of a solve (int[kSzWords]).  A solve replayed from a CUDA
// graph reads every count and level range here instead of from host arguments;
// the kernels that take a nullable `sz` use it when it is given.  When a count
// exceeds a capacity of the plan, the step that finds it sets kSzAbort and
// clamps the count (to zero, or to the last level), so that every later step
// stays inside its buffers; the result of that replay is then invalid.
enum {
    kSzLevel = 0,      // first cell of each level, kMaxLevel + 2 entries
    kSzTileBase = 24,  // first M2L tile of the children of each level's cells
    kSzTiles = 48,     // M2L tiles in use
    kSzCells,          // cells
    kSzLeaves,         // leaves
    kSzClasses,        // offset classes
    kSzEntries,        // (tile, class) blocks
    kSzUnits,          // M2L work units
    kSzAbort,          // nonzero: a plan capacity was exceeded
    kSzWords = 64
};
static_assert(kMaxLevel + 2 <= kSzTileBase - kSzLevel, "level starts overflow their slot");

// Structure-of-arrays cells, level by level (Morton order within a level).
struct CellArrays {
    int *level;
    uint64_t *prefix;  // top 3*level key bits, right-aligned
    int *begin, *end;  // sorted particle range
    int *parent, *child0, *nchild;
    int *tile, *lane;  // M2L GEMM tile of this cell as a target
    int *sys;          // independent system (root) the cell belongs to
    int4 *geom;        // integer centre (x, y, z) in units of side/2^22; w = half side
                       // (bits 0-23) | count bucket of the hybrid selection << 24
    // centre in FP32 as hi + lo parts with 1/side (fhi.w) and side (flo.w): the frame
    // of the expansion kernels' particle offsets, without FP64 per particle
    float4 *fhi, *flo;
};

// Interaction lists written by the traversal (CSR per target cell).
struct ListArrays {
    int *m2l_src;         // source cell per M2L pair
    int *m2l_tgt;         // target cell per M2L pair
    uint32_t *m2l_slot;   // class hash slot, later replaced by the class id
    int *p2p_src, *p2p_tgt;
    int *m2l_off, *m2l_cnt, *p2p_off, *p2p_cnt;  // per cell
    int *def_off, *def_cnt;                      // per cell: deferred sources
    int *def_src;
    int *m2p_src, *m2p_tgt;                      // cell-particle pairs (hybrid value 2)
    int *m2p_off, *m2p_cnt;                      // per cell
    int *p2l_src, *p2l_tgt;                      // particle-cell pairs (hybrid value 3)
    int *p2l_off, *p2l_cnt;                      // per cell
};

constexpr int kHashBits = 18;
constexpr uint32_t kHashCap = 1u << kHashBits;
constexpr uint64_t kHashEmpty = ~0ull;

// The caller's arrays of a replayed plan.  The kernels that read the particles
// or write the results take them from here when io is given (the host writes
// the four pointers before each replay), so that one captured plan serves any
// arrays in place.
struct IoPtrs {
    const float *xyz, *q;
    float *phi, *grad;
};

// tree.cu
__global__ void k_init_bbox(uint32_t *bbox_u, int nsys);
__global__ void k_bbox(const float *xyz, int64_t n, uint32_t *bbox_u, int *flags, const IoPtrs *io = nullptr);
__global__ void k_morton(const float *xyz, int64_t n, const int *off, int nsys,
                         const uint32_t *bbox_u, double *box, uint64_t *keys, uint32_t *idx,
                         const IoPtrs *io = nullptr);
__global__ void k_bbox_sys(const float *xyz, int64_t n, const int *off, int nsys, uint32_t *bbox_u,
                           int *flags, const IoPtrs *io = nullptr);
__global__ void k_sys_of_sorted(const uint32_t *idx, int64_t n, const int *off, int nsys,
                                uint64_t *sys_key);
__global__ void k_gather_keys(const uint64_t *orig, const uint32_t *idx, int64_t n, uint64_t *keys);
__global__ void k_init_roots(CellArrays c, const int *off, int nsys);
__global__ void k_permute(const float *xyz, const float *q, const uint32_t *idx, int64_t n,
                          float4 *out, const IoPtrs *io = nullptr);
__global__ void k_first_diff(const uint64_t *keys, int64_t n, uint64_t *lvl, uint32_t *pos);
constexpr int kLevelStartWarps = 24;  // levels 0 .. 23, one warp each
__global__ void k_level_starts(const uint64_t *lvl, int64_t n, int *start);
// With sz: the level's cells come from sz, packed has len entries (zero past the
// level) and emission stops at the level end sz clamps to.
__global__ void k_split_count(CellArrays c, const uint32_t *bpos, const int *lstart, int a, int b,
                              int level, int ncrit, int max_depth, int64_t *packed, const int *sz = nullptr,
                              int len = 0);
__global__ void k_split_emit(CellArrays c, const uint64_t *keys, const uint32_t *bpos,
                             const int *lstart, int a, int b, int level, const int64_t *packed,
                             const int64_t *ex, int tile_base, const int *sz = nullptr);
// Next level start and tile base from a level's split totals, against the
// plan's capacities (graph replay only).
__global__ void k_level_advance(const int64_t *total, int level, int last_level, int cell_cap,
                                int next_level_cap, int tile_cap, int *sz);
// The first levels of a tree with device-side level ranges, in one block (see tree.cu).
constexpr int kSmallLevelCells = 4096;
constexpr int kSmallLevelThreads = 1024;
constexpr int kMaxSmallLevels = 16;
struct SmallLevels {
    int n;                         // levels 0 .. n - 1 are split by the one block
    int cap[kMaxSmallLevels + 1];  // cell capacity of each level (cap[l + 1]: the children of level l)
};
__global__ void k_tree_small_levels(CellArrays c, const uint64_t *keys, const uint32_t *bpos, const int *bstart,
                                    int ncrit, int max_depth, SmallLevels sl, int last_level, int cell_cap,
                                    int tile_cap, int *sz);
__global__ void k_fill_tile_cells(CellArrays c, int ncells, int *tile_cells, const int *sz = nullptr);
// M2L tiles regrouped by likeness of the targets' class sets (tree.cu): sort
// keys of len cells (past the last cell: a key that sorts last), then, from the
// stably sorted (key, cell) pairs, each cell's tile and lane.  lstart: first
// cell of each level.  With sz: the cell count from sz, and kSzAbort on a tile
// past tile_cap.
__global__ void k_tile_keys(CellArrays c, int ncells, const int *m2l_cnt, int len, uint64_t *key, uint32_t *val,
                            const int *sz = nullptr);
__global__ void k_tile_assign(const uint64_t *key, const uint32_t *val, int ncells, const int *lstart, int tile_cap,
                              CellArrays c, int *sz = nullptr);
constexpr int kTileSortBits = 28;
// c.geom of every cell from its level and key prefix (with sz: the cell count from sz).
__global__ void k_cell_geom(CellArrays c, int ncells, const double *box, const int *sz = nullptr);
// With sz: flags for len cells, zero past the last cell.
__global__ void k_leaf_flags(CellArrays c, int ncells, int *flag, const int *sz = nullptr, int len = 0);
__global__ void k_leaf_compact(CellArrays c, int ncells, const int *ex, int *leaves, const int *sz, int *pcell);

// traverse.cu
constexpr int kSelNB = 128;  // count buckets of the hybrid selection table
// Count bucket of the selection table: n - 1 below 4, then four per octave.
constexpr int kGeomHalfMask = (1 << 24) - 1;
constexpr int kGeomBucketShift = 24;
__device__ __forceinline__ int count_bucket(int n)
{
    const int e = 31 - __clz(n);
    return e < 2 ? n - 1 : 3 + 4 * (e - 2) + ((n >> (e - 2)) & 3);
}
__global__ void k_traverse_level(CellArrays c, ListArrays L, int a, int b, double theta2,
                                 float theta2f, const uint8_t *sel, unsigned long long *counters,
                                 int64_t cap_m, int64_t cap_p, int64_t cap_d, int64_t cap_q,
                                 int64_t cap_l, uint64_t *hash_keys, int *flags, const int *sz = nullptr,
                                 int level = 0);
// List totals against capacities (graph replay): totals[k] = counters[k], or
// zero for every list (and kSzAbort set) when one exceeds its capacity.
__global__ void k_check_lists(const unsigned long long *counters, int64_t cap_m, int64_t cap_p, int64_t cap_d,
                              int64_t cap_q, int64_t cap_l, unsigned long long *totals, int *sz);
// Offset classes against the plan (graph replay): nclass from the hash scan (on
// overflow no class and no M2L pair), then each class key's table slot from the
// plan's key table (open addressing, hcap a power of two); a class the plan has
// no table for sets kSzAbort.
__global__ void k_plan_classes(const int *nclass_dev, int nclass_cap, int *sz, unsigned long long *totals);
__global__ void k_class_lookup(const uint64_t *sorted_keys, const int *sz, const uint64_t *hkeys,
                               const int *hslots, uint32_t hcap, int *class_slot, int *szw);
// Entries against the plan's capacity (graph replay): on overflow every tile is
// emptied and kSzAbort set.  One block.
__global__ void k_check_entries(int *entry_base, int ntiles_cap, int nent_cap, int *sz);
__global__ void k_hash_flags(const uint64_t *hash_keys, int *flag);
__global__ void k_hash_compact(const uint64_t *hash_keys, const int *ex, uint64_t *ukeys,
                               uint32_t *uslot);
__global__ void k_root_lists(CellArrays c, ListArrays L, int nsys, unsigned long long *counters);
__global__ void k_rank_classes(const uint64_t *ukeys, const uint32_t *uslot, int n,
                               uint64_t *sorted_keys, int *slot_class, const int *sz = nullptr);
__global__ void k_slot_to_class(const uint32_t *uslot, int nclass, int *slot_class);
// dn (nullable): the pair count in device memory.
__global__ void k_m2l_class(uint32_t *m2l_slot, int64_t n, const int *slot_class,
                            const unsigned long long *dn = nullptr);
__global__ void k_tile_bitmap(const int *m2l_tgt, const uint32_t *m2l_class, int64_t n,
                              const int *cell_tile, int nwords, uint32_t *bitmap,
                              const unsigned long long *dn = nullptr);
__global__ void k_tile_popc(const uint32_t *bitmap, int ntiles, int nwords, int *cnt);
__global__ void k_tile_entries(const uint32_t *bitmap, int ntiles, int nwords,
                               const int *entry_base, int *word_prefix, int *entry_class,
                               const int *class_slot, int entry_cap = INT_MAX);
// src[entry * kTile + row] = source cell of each M2L pair, written row by row in
// tile order (a warp per row; with sz, the tile count from sz), so that the
// writes in flight stay within a few tiles' entries.
__global__ void k_tile_src_rows(const int *tile_cells, int ntiles, const int *m2l_off, const int *m2l_cnt,
                                const int *m2l_src, const uint32_t *m2l_class, int nwords, const uint32_t *bitmap,
                                const int *word_prefix, int *src, const int *sz = nullptr, int entry_cap = INT_MAX);

// expansions.cu
__global__ void k_build_m2l_tables(const uint64_t *class_keys, const int *cache_slot, int nnew,
                                   int p, int P2pad, float *table);
__global__ void k_build_shift_tables(int p, int P2pad, float *m2m, float *l2l, double *m2m64, double *l2l64);
// P2M, one warp (32-thread block) per leaf of leaves[0, nleaves), grid blocks;
// an instantiation with the order fixed at compile time for p = 4, 6, 8, 10, 12.
void launch_p2m(const CellArrays &c, const int *leaves, int nleaves, unsigned grid, const float4 *pts, int p,
                int P2pad, float *M, cudaStream_t st, const int *sz = nullptr);
// Fills the recurrence-coefficient tables P2M and L2P read (once per device).
void init_recurrence_tables();
// M2M (l2l = false: parents [a, b) of E from their children, through the
// per-child scratch T[ncells][P2pad]) or L2L (l2l = true: the children of
// parents [a, b) of E from them), octant-batched.
// With sz: parents are the cells of `level` in sz, launched for up to `cap`
// of them (a and b are ignored).
void launch_shift_batched(bool l2l, const CellArrays &c, int a, int b, const float *mats, int P2, int P2pad,
                          float *E, float *T, cudaStream_t st, const int *sz = nullptr, int level = 0,
                          int cap = 0);
// The same shifts with FP64 matrices and sums, for the top levels at high p.
constexpr int kFp64TopP = 12, kFp64TopLevels = 3;  // p >= 12: parents at levels 0..2
void launch_shift_fp64(bool l2l, const CellArrays &c, int a, int b, const double *mats, int P2, int P2pad, float *E,
                       cudaStream_t st, const int *sz = nullptr, int level = 0, int cap = 0);
// L2P, particle-parallel: warps of 32 consecutive sorted particles, pcell[i] =
// the leaf of sorted particle i (k_leaf_compact), n particles.
void launch_l2p(const CellArrays &c, const int *pcell, int64_t n, const float4 *pts, int p, int P2pad,
                const float *L, float4 *far, cudaStream_t st);
// Shared memory of one leaf's L2P records: one 32-byte record per term (n, m),
// m <= n <= p, then the leaf's P2pad coefficients.
inline size_t l2p_smem(int p, int P2pad) { return (size_t)(p + 1) * (p + 2) / 2 * 32 + (size_t)P2pad * 4; }
// P2L: one warp (block) per target cell with a P2L list; the source particles are
// added to the cell's local expansion.  Dynamic shared memory 32 (P2pad + 1) floats.
__global__ void k_p2l(CellArrays c, ListArrays Ls, int ncells, const float4 *pts, const double *box, int p,
                      int P2pad, float *L, const int *sz = nullptr);
// M2P: blocks of kM2PWarps warps, one target leaf per warp; dynamic shared memory m2p_smem(p, P2pad).
constexpr int kM2PWarps = 4;
size_t m2p_smem(int p, int P2pad);
__global__ void k_m2p(CellArrays c, ListArrays Ls, const int *leaves, int nleaves, const float4 *pts,
                      const double *box, int p, int P2pad, const float *M, float4 *far, const int *sz = nullptr);

// m2l.cu
void launch_m2l_simt(int ntiles, const int *entry_base, const int *entry_class, const int *src,
                     const int *tile_cells, const float *M, const float *table, int P2pad,
                     float *L, cudaStream_t st);

// m2l_tc.cu
struct M2LUnit {
    int tile, e0, e1, pad;
};
bool m2l_tc_supported(int P2pad);
// One bounded wait on an mbarrier nothing arrives at (failure-detection self-test).
void launch_wait_selftest(uint32_t polls, int *flags, cudaStream_t st);
size_t m2l_tc_smem(int P2pad, bool bf16, int &nstages);
// With sz: launched for nunits (a capacity) units, of which the first sz[kSzUnits] run.
void launch_m2l_tc(bool bf16, int nunits, const void *units, int ntiles, const int *unit_base,
                   const int *tile_units, const int *entry_class, const int *src, const int *tile_cells,
                   const float *M, const unsigned char *tsplit, int P2pad, float *partial, float *L,
                   int *flags, cudaStream_t st, const int *sz = nullptr);
// Work units: per tile ceil(blocks / chunk) units of chunk blocks, the last one
// shorter.  Execution order: the full units by (rank within the tile, tile), then
// the shorter last units by size class (kUnitBuckets classes, longer first).
constexpr int kUnitBuckets = 8;
// Work units on the device (graph replay), as the host builds them; kSzAbort and
// no units when more than units_cap would be needed.  One block.
__global__ void k_build_units(const int *entry_base, int ntiles_cap, int chunk, int units_cap, M2LUnit *units,
                              int *unit_base, int *tile_units, int *sz);
// Bytes of the hi/lo split class matrices of nslots classes, and the kernel that
// writes slots [slot0, slot0 + nslots) of them from the FP32 tables.
size_t m2l_split_bytes(int P2pad, bool bf16, int nslots);
void launch_split_tables(bool bf16, const float *table, int slot0, int nslots, int P2pad, unsigned char *out,
                         cudaStream_t st);

// p2p.cu -- P2P: one 32-thread block per target leaf (grid >= nleaves), up to
// kP2PWarpsPerSM resident per SM; the FP32 ceiling probe of the interaction body
// runs kP2PBlocksPerSM blocks of 128 threads per SM (the same warps per SM)
constexpr int kP2PWarpsPerSM = 16;
constexpr int kP2PBlocksPerSM = 4;
__global__ void k_p2p(CellArrays c, ListArrays L, const int *leaves, int nleaves,
                      const float4 *pts, float4 *near, const int *sz = nullptr);
__global__ void k_direct(const float *xyz, const float *q, int64_t n, float *phi, float *grad);
// FP32-pipe ceilings: FP32x2 FMA chains (16 lane-FMAs per thread and iteration),
// and the P2P interaction body on staged sources (32 interactions per thread and rep).
__global__ void k_ffma_stream(float *out, int iters, float s);
__global__ void k_p2p_body(float *out, int reps);
__global__ void k_combine(const float4 *far, const float4 *near, const uint32_t *idx, int64_t n,
                          float *phi, float *grad, const IoPtrs *io = nullptr);

// mlp.cu -- cost-model network (3 layers, hidden 64, FP16 parameters)
constexpr int kMlpIn = 4, kMlpHidden = 64, kMlpOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpHidden * kMlpIn, kOffW2 = kOffB1 + kMlpHidden,
              kOffB2 = kOffW2 + kMlpHidden * kMlpHidden, kOffW3 = kOffB2 + kMlpHidden,
              kOffB3 = kOffW3 + kMlpOut * kMlpHidden, kMlpParams = kOffB3 + kMlpOut;
size_t mlp_grad_smem();
__global__ void k_mlp_forward(const __half *w16, const float *x, int B, float *y);
__global__ void k_mlp_grad_partial(const __half *w16, const float *x, const float *t, const float *m, int B,
                                   const float *inv_cnt, float *partial, float *loss_part);
__global__ void k_mlp_mask_count(const float *m, int n, float *inv_cnt);
__global__ void k_mlp_reduce(const float *partial, int nblk, const float *loss_part, float *grad,
                             float *loss);
__global__ void k_mlp_adam(float *w32, float *mom, float *vel, const float *g, __half *w16, int *step,
                           float lr, float beta1, float beta2, float eps);
__global__ void k_mlp_step_inc(int *step);
__global__ void k_mlp_table(const __half *w16, float p, float sep, uint8_t *sel);
__global__ void k_pair_bucket_hist(const int *tgt, const int *src, int64_t n, const int *begin, const int *end,
                                   unsigned long long *hist);
__global__ void k_mlp_solve_cost(const __half *w16, float p, float sep, const unsigned long long *hist,
                                 unsigned long long m2l_pairs, double *out);

// cost_model.cu -- kernel pre-calculation on artificial cells
struct P2PTiming {
    int nt, ns;          // particles per target leaf and per source cell
    double ns_per_pair;  // device time per (target leaf, source cell) pair
};
// Times the P2P kernel on artificial leaves for every (nt, ns) in counts x counts.
std::vector<P2PTiming> pretime_p2p(const std::vector<int> &counts, uint64_t seed, cudaStream_t st);
// M2P time per (target leaf, source cell) pair at expansion order p for each
// target count in counts.
std::vector<double> pretime_m2p(int p, const std::vector<int> &counts, uint64_t seed, cudaStream_t st);
// P2L time per (target cell, source cell) pair at order p for each source count in counts.
std::vector<double> pretime_p2l(int p, const std::vector<int> &counts, uint64_t seed, cudaStream_t st);
// Selection table: the cheapest of M2L (m2l_ns per pair), P2P (interpolated from
// the grid), M2P (interpolated over the target count) and P2L (over the source
// count); M2P or P2L is not considered when its timings are empty.
void table_from_timings(const std::vector<P2PTiming> &grid, double m2l_ns, const std::vector<int> &m2p_counts,
                        const std::vector<double> &m2p_ns, const std::vector<double> &p2l_ns, uint8_t *sel);
// log2 of the representative count of a selection-table bucket (host and device agree).
__host__ __device__ inline float bucket_mid_log2(int b)
{
    if (b < 3) return log2f((float)(b + 1));
    const int e = (b - 3) / 4 + 2, k = (b - 3) % 4;
    const float lo = ldexpf(1.f + 0.25f * k, e), hi = ldexpf(1.f + 0.25f * (k + 1), e) - 1.f;
    return 0.5f * (log2f(lo) + log2f(hi > lo ? hi : lo));
}

}  // namespace fmm
