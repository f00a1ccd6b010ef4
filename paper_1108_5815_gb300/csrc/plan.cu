// plan.cu -- the solve of a plan, issued without host read-backs so that it can
// be captured into one CUDA graph (one graph launch solves every system of the
// plan).  The steps and kernels are those of the plain solve in fmm_api.cu; the
// differences are that every count and level range comes from the device sizes
// block, every launch is sized by the plan's capacity, and a step that finds a
// count above its capacity marks the replay invalid instead of regrowing.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace fmm {

__global__ void k_plan_init(int *__restrict__ sz, int nsys)
{
    for (int i = threadIdx.x; i < kSzWords; i += blockDim.x) sz[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        sz[kSzLevel + 0] = 0;
        sz[kSzLevel + 1] = nsys;
        sz[kSzTiles] = (nsys + kTile - 1) / kTile;  // the roots' tiles
        sz[kSzCells] = nsys;
    }
}

namespace {

unsigned blocks_for(int64_t n, int per) { return (unsigned)std::max<int64_t>(1, ceil_div(n, per)); }

// the grid the plain solve uses for its grid-stride kernels
unsigned grid_stride(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 152 * 16)); }

}  // namespace

void enqueue_plan(const PlanShape &s, const PlanBuffers &b, cudaStream_t st, cudaStream_t fs, cudaEvent_t tree,
                  cudaEvent_t fork, cudaEvent_t join)
{
    const int N = s.N, nsys = s.nsys;
    const CellArrays &c = b.c;
    const ListArrays &L = b.L;

    // ---------------------------------------------------------- box, keys, sort
    FMM_CUDA_TRY(cudaMemsetAsync(b.flags, 0, sizeof(int) * kNumFlags, st));
    k_plan_init<<<1, 64, 0, st>>>(b.sz, nsys);
    FMM_LAUNCH_CHECK();
    k_init_bbox<<<blocks_for(6 * (int64_t)nsys, 256), 256, 0, st>>>(b.bbox_u, nsys);
    FMM_LAUNCH_CHECK();
    if (nsys == 1)
        k_bbox<<<grid_stride(N), 256, 0, st>>>(b.xyz, N, b.bbox_u, b.flags, b.io);
    else
        k_bbox_sys<<<blocks_for(ceil_div(N, 8), 256), 256, 0, st>>>(b.xyz, N, b.sys_off, nsys, b.bbox_u, b.flags,
                                                                    b.io);
    FMM_LAUNCH_CHECK();
    k_morton<<<grid_stride(N), 256, 0, st>>>(b.xyz, N, b.sys_off, nsys, b.bbox_u, b.box, b.keys, b.idx, b.io);
    FMM_LAUNCH_CHECK();
    if (nsys == 1) {
        radix_sort_pairs(b.keys, b.idx, b.keys_alt, b.idx_alt, N, 63, b.hist, b.flags, st);
    } else {
        FMM_CUDA_TRY(cudaMemcpyAsync(b.keys_orig, b.keys, sizeof(uint64_t) * N, cudaMemcpyDeviceToDevice, st));
        radix_sort_pairs(b.keys, b.idx, b.keys_alt, b.idx_alt, N, 63, b.hist, b.flags, st);
        k_sys_of_sorted<<<grid_stride(N), 256, 0, st>>>(b.idx, N, b.sys_off, nsys, b.sys_key);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(b.sys_key, b.idx, b.keys_alt, b.idx_alt, N, s.sys_bits, b.hist, b.flags, st);
        k_gather_keys<<<grid_stride(N), 256, 0, st>>>(b.keys_orig, b.idx, N, b.keys);
        FMM_LAUNCH_CHECK();
    }
    k_permute<<<grid_stride(N), 256, 0, st>>>(b.xyz, b.q, b.idx, N, b.pts, b.io);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- tree
    k_init_roots<<<blocks_for(nsys, 256), 256, 0, st>>>(c, b.sys_off, nsys);
    FMM_LAUNCH_CHECK();
    if (N > 1) {
        k_first_diff<<<grid_stride(N), 256, 0, st>>>(b.keys, N, b.blvl, b.bpos);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(b.blvl, b.bpos, b.keys_alt, b.idx_alt, N - 1, 8, b.hist, b.flags, st);
    }
    k_level_starts<<<1, 32 * kLevelStartWarps, 0, st>>>(b.blvl, N - 1, b.bstart);
    FMM_LAUNCH_CHECK();
    // the first levels whose capacities are small: one block splits them all
    int nsmall = 0;
    while (nsmall < kMaxSmallLevels && nsmall <= s.levels && s.level_cap[nsmall] <= kSmallLevelCells) ++nsmall;
    if (nsmall > 0) {
        SmallLevels sl{};
        sl.n = nsmall;
        for (int l = 0; l <= nsmall; ++l) sl.cap[l] = s.level_cap[l];
        k_tree_small_levels<<<1, kSmallLevelThreads, 0, st>>>(c, b.keys, b.bpos, b.bstart, s.ncrit, s.max_depth, sl,
                                                                s.levels, s.cell_cap, s.tile_cap, b.sz);
        FMM_LAUNCH_CHECK();
    }
    for (int l = nsmall; l <= s.levels; ++l) {
        const int len = s.level_cap[l];
        k_split_count<<<blocks_for(len, 128), 128, 0, st>>>(c, b.bpos, b.bstart, 0, 0, l, s.ncrit, s.max_depth,
                                                            b.packed, b.sz, len);
        FMM_LAUNCH_CHECK();
        scan_exclusive<int64_t>(b.packed, b.packed_ex, len, b.packed_ex + len, b.scan_i64, st);
        k_level_advance<<<1, 1, 0, st>>>(b.packed_ex + len, l, s.levels, s.cell_cap, s.level_cap[l + 1], s.tile_cap,
                                         b.sz);
        FMM_LAUNCH_CHECK();
        k_split_emit<<<blocks_for(len, 128), 128, 0, st>>>(c, b.keys, b.bpos, b.bstart, 0, 0, l, b.packed,
                                                           b.packed_ex, 0, b.sz);
        FMM_LAUNCH_CHECK();
    }
    k_leaf_flags<<<blocks_for(s.cell_cap, 256), 256, 0, st>>>(c, 0, b.leaf_flag, b.sz, s.cell_cap);
    FMM_LAUNCH_CHECK();
    scan_exclusive<int>(b.leaf_flag, b.leaf_ex, s.cell_cap, b.leaf_ex + s.cell_cap, b.scan_i32, st);
    k_leaf_compact<<<blocks_for(s.cell_cap, 256), 256, 0, st>>>(c, 0, b.leaf_ex, b.leaves, b.sz, b.pcell);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaMemcpyAsync(b.sz + kSzLeaves, b.leaf_ex + s.cell_cap, sizeof(int), cudaMemcpyDeviceToDevice, st));
    k_cell_geom<<<grid_stride(s.cell_cap), 256, 0, st>>>(c, 0, b.box, b.sz);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- upward pass (fs, beside the traversal)
    const int p = s.p, P2 = s.P2, P2pad = s.P2pad;
    FMM_CUDA_TRY(cudaEventRecord(tree, st));
    FMM_CUDA_TRY(cudaStreamWaitEvent(fs, tree, 0));
    launch_p2m(c, b.leaves, 0, (unsigned)std::max(1, s.leaf_cap), b.pts, p, P2pad, b.M, fs, b.sz);
    for (int l = s.levels - 1; l >= 0; --l) {
        if (p >= kFp64TopP && l < kFp64TopLevels)
            launch_shift_fp64(false, c, 0, 0, b.m2m64, P2, P2pad, b.M, fs, b.sz, l, s.level_cap[l]);
        else
            launch_shift_batched(false, c, 0, 0, b.m2m, P2, P2pad, b.M, b.mtmp, fs, b.sz, l, s.level_cap[l]);
    }

    // ---------------------------------------------------------- traversal
    const double theta2 = s.theta * s.theta;
    FMM_CUDA_TRY(cudaMemsetAsync(b.hash_keys, 0xff, sizeof(uint64_t) * kHashCap, st));
    k_root_lists<<<1, 256, 0, st>>>(c, L, nsys, b.tcount);
    FMM_LAUNCH_CHECK();
    for (int l = 1; l <= s.levels; ++l) {
        k_traverse_level<<<blocks_for((int64_t)s.level_cap[l] * 32, 128), 128, 0, st>>>(
            c, L, 0, 0, theta2, (float)theta2, b.sel, b.tcount, s.m2l_cap, s.p2p_cap, s.def_cap, s.m2p_cap,
            s.p2l_cap, b.hash_keys, b.flags, b.sz, l);
        FMM_LAUNCH_CHECK();
    }
    k_check_lists<<<1, 1, 0, st>>>(b.tcount, s.m2l_cap, s.p2p_cap, s.def_cap, s.m2p_cap, s.p2l_cap, b.totals, b.sz);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- fork: P2P on st
    FMM_CUDA_TRY(cudaEventRecord(fork, st));
    FMM_CUDA_TRY(cudaStreamWaitEvent(fs, fork, 0));
    k_p2p<<<(unsigned)std::max(1, s.leaf_cap), 32, 0, st>>>(c, L, b.leaves, 0, b.pts, b.near, b.sz);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- M2L tiles regrouped (fs, tensor-core M2L)
    if (s.tensor) {
        k_tile_keys<<<grid_stride(s.cell_cap), 256, 0, fs>>>(c, 0, L.m2l_cnt, s.cell_cap, b.tile_key, b.tile_val,
                                                             b.sz);
        FMM_LAUNCH_CHECK();
        radix_sort_pairs(b.tile_key, b.tile_val, b.tile_key_alt, b.tile_val_alt, s.cell_cap, kTileSortBits,
                         b.tile_hist, b.flags, fs);
        k_tile_assign<<<grid_stride(s.cell_cap), 256, 0, fs>>>(b.tile_key, b.tile_val, 0, b.sz + kSzLevel,
                                                               s.tile_cap, c, b.sz);
        FMM_LAUNCH_CHECK();
    }

    // ---------------------------------------------------------- offset classes (fs)
    k_hash_flags<<<kHashCap / 256, 256, 0, fs>>>(b.hash_keys, b.hflag);
    FMM_LAUNCH_CHECK();
    scan_exclusive<int>(b.hflag, b.hex, kHashCap, b.hex + kHashCap, b.scan_i32, fs);
    k_plan_classes<<<1, 1, 0, fs>>>(b.hex + kHashCap, s.nclass_cap, b.sz, b.totals);
    FMM_LAUNCH_CHECK();
    k_hash_compact<<<kHashCap / 256, 256, 0, fs>>>(b.hash_keys, b.hex, b.ukeys, b.uslot);
    FMM_LAUNCH_CHECK();
    k_rank_classes<<<blocks_for(s.nclass_cap, 128), 128, 0, fs>>>(b.ukeys, b.uslot, 0, b.ukeys_alt, b.slot_class,
                                                                  b.sz);
    FMM_LAUNCH_CHECK();
    k_class_lookup<<<blocks_for(s.nclass_cap, 128), 128, 0, fs>>>(b.ukeys_alt, b.sz, b.chash_keys, b.chash_slots,
                                                                  s.class_hcap, b.class_slot, b.sz);
    FMM_LAUNCH_CHECK();
    k_m2l_class<<<grid_stride(s.m2l_cap), 256, 0, fs>>>(L.m2l_slot, 0, b.slot_class, b.totals);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- M2L tiles (fs)
    FMM_CUDA_TRY(cudaMemsetAsync(b.tile_cells, 0xff, sizeof(int) * (size_t)s.tile_cap * kTile, fs));
    FMM_CUDA_TRY(cudaMemsetAsync(b.bitmap, 0, sizeof(uint32_t) * (size_t)s.tile_cap * s.nwords, fs));
    k_fill_tile_cells<<<blocks_for(s.cell_cap, 256), 256, 0, fs>>>(c, 0, b.tile_cells, b.sz);
    FMM_LAUNCH_CHECK();
    k_tile_bitmap<<<grid_stride(s.m2l_cap), 256, 0, fs>>>(L.m2l_tgt, L.m2l_slot, 0, c.tile, s.nwords, b.bitmap,
                                                          b.totals);
    FMM_LAUNCH_CHECK();
    k_tile_popc<<<blocks_for(s.tile_cap, 4), 128, 0, fs>>>(b.bitmap, s.tile_cap, s.nwords, b.tile_cnt);
    FMM_LAUNCH_CHECK();
    scan_exclusive<int>(b.tile_cnt, b.entry_base, s.tile_cap, b.entry_base + s.tile_cap, b.scan_i32, fs);
    k_check_entries<<<1, 256, 0, fs>>>(b.entry_base, s.tile_cap, s.nent_cap, b.sz);
    FMM_LAUNCH_CHECK();
    k_tile_entries<<<blocks_for(s.tile_cap, 4), 128, 0, fs>>>(b.bitmap, s.tile_cap, s.nwords, b.entry_base,
                                                              b.word_prefix, b.entry_class, b.class_slot,
                                                              s.nent_cap);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaMemsetAsync(b.src, 0xff, sizeof(int) * (size_t)s.nent_cap * kTile, fs));
    k_tile_src_rows<<<blocks_for((int64_t)s.tile_cap * kTile, 4), 128, 0, fs>>>(
        b.tile_cells, 0, L.m2l_off, L.m2l_cnt, L.m2l_src, L.m2l_slot, s.nwords, b.bitmap, b.word_prefix, b.src, b.sz,
        s.nent_cap);
    FMM_LAUNCH_CHECK();

    // ---------------------------------------------------------- M2L (fs)
    if (s.tensor) {
        k_build_units<<<1, 1024, 0, fs>>>(b.entry_base, s.tile_cap, s.chunk, s.units_cap, b.units, b.unit_base,
                                          b.tile_units, b.sz);
        FMM_LAUNCH_CHECK();
        launch_m2l_tc(s.bf16, s.units_cap, b.units, s.tile_cap, b.unit_base, b.tile_units, b.entry_class, b.src,
                      b.tile_cells, b.M, b.tsplit, P2pad, b.partial, b.Lx, b.flags, fs, b.sz);
    } else {
        launch_m2l_simt(s.tile_cap, b.entry_base, b.entry_class, b.src, b.tile_cells, b.M, b.table, P2pad, b.Lx, fs);
    }

    // ---------------------------------------------------------- downward pass (fs)
    if (s.p2l_seen) {  // particle-cell pairs (the plan has none of a kind its capture lacked)
        k_p2l<<<(unsigned)std::max(1, s.cell_cap), 32, (size_t)32 * (P2pad + 1) * sizeof(float), fs>>>(
            c, L, 0, b.pts, b.box, p, P2pad, b.Lx, b.sz);
        FMM_LAUNCH_CHECK();
    }
    for (int l = 0; l < s.levels; ++l) {
        if (p >= kFp64TopP && l < kFp64TopLevels)
            launch_shift_fp64(true, c, 0, 0, b.l2l64, P2, P2pad, b.Lx, fs, b.sz, l, s.level_cap[l]);
        else
            launch_shift_batched(true, c, 0, 0, b.l2l, P2, P2pad, b.Lx, nullptr, fs, b.sz, l, s.level_cap[l]);
    }
    launch_l2p(c, b.pcell, s.N, b.pts, p, P2pad, b.Lx, b.far, fs);
    if (s.m2p_seen) {  // cell-particle pairs
        k_m2p<<<blocks_for(s.leaf_cap, kM2PWarps), 32 * kM2PWarps, m2p_smem(p, P2pad), fs>>>(
            c, L, b.leaves, 0, b.pts, b.box, p, P2pad, b.M, b.far, b.sz);
        FMM_LAUNCH_CHECK();
    }

    // ---------------------------------------------------------- join and combine
    FMM_CUDA_TRY(cudaEventRecord(join, fs));
    FMM_CUDA_TRY(cudaStreamWaitEvent(st, join, 0));
    k_combine<<<grid_stride(N), 256, 0, st>>>(b.far, b.near, b.idx, N, b.phi, b.grad, b.io);
    FMM_LAUNCH_CHECK();
}

}  // namespace fmm
