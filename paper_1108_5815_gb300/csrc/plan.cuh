// plan.cuh -- a solve with every size on the device, for CUDA-graph capture.
//
// A plan fixes N, the systems, p, theta, ncrit and the options, and gives every
// buffer a capacity (the sizes of a first solve with headroom).  enqueue_plan
// issues the whole solve -- keys, sort, tree, traversal, P2P, classes, tiles,
// upward pass, M2L, downward pass, combine -- without one host read-back: each
// kernel reads its counts and level ranges from the device sizes block
// (kSzWords ints), launched for the capacity.  A step that finds a count above
// its capacity, or an offset class with no operator in the plan, sets kSzAbort
// and clamps the counts so that every later step stays inside its buffers; the
// caller reads the status after the replay and makes a new plan.
#pragma once

#include <string>
#include <vector>

#include "kernels.cuh"

namespace fmm {

struct PlanShape {
    int N = 0, nsys = 1, p = 0, P2 = 0, P2pad = 0, ncrit = 0, max_depth = 0;
    double theta = 0.0;
    bool tensor = false, bf16 = false;  // M2L on the tensor cores, BF16x3 (else TF32x3)
    bool hybrid = false;                // a selection table is in use (M2P/P2L possible)
    bool m2p_seen = false, p2l_seen = false;  // the captured solve had such pairs (else none allowed)
    int sys_bits = 1;                   // bits of the system index (batched sort)
    int levels = 0;                     // parents at levels 0 .. levels - 1; level `levels` must not split
    std::vector<int> level_cap;         // cells per level, levels + 2 entries
    int cell_cap = 0, leaf_cap = 0, tile_cap = 0, nclass_cap = 0, nent_cap = 0, units_cap = 0;
    int chunk = 8, nwords = 1, nsm = 152;
    int64_t m2l_cap = 0, p2p_cap = 0, def_cap = 0, m2p_cap = 0, p2l_cap = 0;
    uint32_t class_hcap = 1;  // size of the class-key table (a power of two)
    int max_level_cap = 0;    // largest entry of level_cap
};

struct PlanBuffers {
    const float *xyz = nullptr, *q = nullptr;  // plan-owned inputs
    float *phi = nullptr, *grad = nullptr;     // plan-owned outputs
    const IoPtrs *io = nullptr;                // or, when set, the caller's arrays (device copy)
    int *flags = nullptr, *sz = nullptr;
    uint32_t *bbox_u = nullptr;
    double *box = nullptr;
    int *sys_off = nullptr;
    uint64_t *keys = nullptr, *keys_alt = nullptr, *keys_orig = nullptr, *sys_key = nullptr;
    uint32_t *idx = nullptr, *idx_alt = nullptr, *hist = nullptr;  // hist: the radix sort scratch
    float4 *pts = nullptr;
    CellArrays c{};
    uint64_t *blvl = nullptr;
    uint32_t *bpos = nullptr;
    int *bstart = nullptr;
    int64_t *packed = nullptr, *packed_ex = nullptr, *scan_i64 = nullptr;
    int *leaf_flag = nullptr, *leaf_ex = nullptr, *scan_i32 = nullptr, *leaves = nullptr;
    int *pcell = nullptr;  // the leaf of each sorted particle (L2P)
    ListArrays L{};
    uint64_t *hash_keys = nullptr;
    unsigned long long *tcount = nullptr, *totals = nullptr;
    const uint8_t *sel = nullptr;
    float4 *far = nullptr, *near = nullptr;
    int *hflag = nullptr, *hex = nullptr;
    uint64_t *ukeys = nullptr, *ukeys_alt = nullptr;
    uint32_t *uslot = nullptr;
    int *slot_class = nullptr, *class_slot = nullptr;
    const uint64_t *chash_keys = nullptr;
    const int *chash_slots = nullptr;
    const float *m2m = nullptr, *l2l = nullptr;
    const double *m2m64 = nullptr, *l2l64 = nullptr;
    const float *table = nullptr;
    const unsigned char *tsplit = nullptr;
    int *tile_cells = nullptr, *tile_cnt = nullptr, *entry_base = nullptr, *word_prefix = nullptr;
    uint64_t *tile_key = nullptr, *tile_key_alt = nullptr;  // the tile regrouping sort (cell_cap pairs)
    uint32_t *tile_val = nullptr, *tile_val_alt = nullptr, *tile_hist = nullptr;
    int *entry_class = nullptr, *src = nullptr;
    uint32_t *bitmap = nullptr;
    M2LUnit *units = nullptr;
    int *unit_base = nullptr, *tile_units = nullptr;
    float *partial = nullptr, *M = nullptr, *Lx = nullptr, *mtmp = nullptr;
};

// Device memory of a plan, freed with it.
struct PlanMemory {
    std::vector<void *> blocks;
    template <typename T>
    T *get(size_t n)
    {
        void *p = nullptr;
        const size_t bytes = (n > 0 ? n : 1) * sizeof(T);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{FMM_ERR_NOMEM, std::string("plan allocation of ") + std::to_string(bytes) + " bytes: " +
                                           cudaGetErrorString(e)};
        }
        blocks.push_back(p);
        return static_cast<T *>(p);
    }
    PlanMemory() = default;
    PlanMemory(const PlanMemory &) = delete;
    PlanMemory &operator=(const PlanMemory &) = delete;
    ~PlanMemory()
    {
        for (void *p : blocks) cudaFree(p);
    }
};

// Enqueues one solve of the plan: st runs the tree, traversal and P2P, fs the
// far-field chain; fork/join order fs after the traversal and st after fs.
void enqueue_plan(const PlanShape &s, const PlanBuffers &b, cudaStream_t st, cudaStream_t fs, cudaEvent_t tree,
                  cudaEvent_t fork, cudaEvent_t join);

// Zeroes the sizes block and sets the roots: level 0 = [0, nsys), tiles of the roots.
__global__ void k_plan_init(int *sz, int nsys);

}  // namespace fmm
