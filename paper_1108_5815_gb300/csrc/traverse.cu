// traverse.cu -- dual tree traversal on the GPU and the M2L offset-class tiles.
//
// The paper's traversal (section "Dual tree traversal") pops (target, source)
// pairs from a LIFO stack, splits the larger cell, and for every new pair
// either evaluates it (far: MAC accepted -> cell-cell; both leaves ->
// particle-particle) or pushes it back.  The fate of a pair depends only on
// the pair, so the same set of interactions is produced by processing targets
// level by level: a target T receives from its parent the sources that were
// pending with the decision "split the target" (the paper: "target cells
// inherit a unique stack of source cells from their parents"), and resolves
// each inherited source S by
//     interact(T,S): MAC -> M2L (or P2P, by the hybrid selection table);
//                    else T,S leaves -> P2P;
//                    else split S (S larger, or T a leaf) and interact with
//                    its children, or defer S to T's children.
// A P2P or M2P pair (T,S) chosen by the selection table above the leaf level is
// handed down as a flagged deferred source until it reaches T's leaves, so the
// P2P and M2P lists stay per-leaf lists (their sources may be cells of any level).
// One warp handles one target; lanes take inherited sources in order and
// resolve each with a small depth-first stack.  Each target's outputs are
// written contiguously in a deterministic order (count, reserve with one atomic
// per list, write), so every per-target list is reproducible.
//
// MAC (reading R3 of the oracle): r = half side, accept iff R > 0 and
// (r_t + r_s)^2 <= theta^2 R^2, evaluated in integer units of side/2^22 so the
// decision is exact and identical to an FP64 CPU evaluation.
#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

constexpr int kStack = 192;
constexpr int kP2PFlag = 1 << 30;  // deferred source that is a chosen P2P pair
constexpr int kM2PFlag = 1 << 29;  // deferred source that is a chosen M2P pair
constexpr int kCellMask = kM2PFlag - 1;
constexpr int kFrontier = 512;  // sources of a leaf target split warp-wide before the walks
constexpr int kCountCache = 32;  // sources whose counts the write pass reuses
// The single pair of a source that is not split (frontier, selection tables):
// M2L, P2P, deferred as it is, M2P, P2L, or deferred with the P2P or M2P flag.
enum { kOutM2L = 0, kOutP2P, kOutDef, kOutM2P, kOutP2L, kOutDefP2P, kOutDefM2P, kOutKinds };

struct TargetInfo {
    int t, level;
    bool leaf;
    int C[3], h;  // centre in units of side/2^22 and half side (< 2^23)
    int bt;       // count bucket of the target (hybrid selection)
};

// Integer centre and half side of cell S (computed once per solve by
// k_cell_geom); its level follows from the half side h = 2^(kKeyBits - level).
// The count bucket of the cell (hybrid selection) rides in the top bits.
__device__ __forceinline__ void cell_geom(const CellArrays &c, int S, int C[3], int &h, int &level, int &bucket)
{
    const int4 g = __ldg(&c.geom[S]);
    C[0] = g.x;
    C[1] = g.y;
    C[2] = g.z;
    h = g.w & kGeomHalfMask;
    level = kKeyBits + 1 - __ffs(h);
    bucket = (int)((unsigned)g.w >> kGeomBucketShift);
}
__device__ __forceinline__ void cell_geom(const CellArrays &c, int S, int C[3], int &h, int &level)
{
    int bucket;
    cell_geom(c, S, C, h, level, bucket);
}

// MAC of reading R3: accept iff R > 0 and (r_t + r_s)^2 <= theta^2 R^2 with theta^2 R^2
// rounded once in FP64.  An FP32 estimate decides every pair farther than a 1e-5
// relative margin from the threshold; the rest take the FP64 comparison itself.
__device__ __forceinline__ bool mac_accept(const TargetInfo &T, const int Cs[3], int hs,
                                           double theta2, float theta2f)
{
    const int dx = T.C[0] - Cs[0], dy = T.C[1] - Cs[1], dz = T.C[2] - Cs[2];
    if ((dx | dy | dz) == 0) return false;
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float r2f = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
    const float rs = (float)(T.h + hs);
    const float lhs = rs * rs, rhs = theta2f * r2f;
    if (lhs < rhs * (1.0f - 1e-5f)) return true;
    if (lhs > rhs * (1.0f + 1e-5f)) return false;
    const int64_t R2 = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
    const int64_t r = (int64_t)T.h + hs;
    return (double)(r * r) <= __dmul_rn(theta2, (double)R2);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ uint32_t hash_insert(uint64_t *table, uint64_t key, int *flags)
{
    uint32_t h = (uint32_t)mix64(key) & (kHashCap - 1);
    for (uint32_t probe = 0; probe < kHashCap; ++probe) {
        uint64_t cur = table[h];
        if (cur == key) return h;
        if (cur == kHashEmpty) {
            uint64_t old = atomicCAS((unsigned long long *)&table[h], (unsigned long long)kHashEmpty,
                                     (unsigned long long)key);
            if (old == kHashEmpty || old == key) return h;
        }
        h = (h + 1) & (kHashCap - 1);
    }
    atomicOr(&flags[kFlagHashFull], 1);
    return 0;
}

// Offset class of an accepted pair: level difference and the centre offset in
// units of the finer cell's half side.
__device__ __forceinline__ uint64_t class_key(const TargetInfo &T, int ls, const int Cs[3],
                                              int *flags)
{
    const int lf = max(T.level, ls);
    const int sh = kKeyBits - lf;  // offsets are exact multiples of 2^sh
    uint64_t key = (uint64_t)(ls - T.level + 64) << 57;
    const int lim = 1 << 18;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int d = (T.C[a] - Cs[a]) >> sh;
        if (d <= -lim || d >= lim) atomicOr(&flags[kFlagClassRange], 1);
        key |= (uint64_t)((d + lim) & 0x7ffff) << (38 - 19 * a);
    }
    return key;
}

struct Counts {
    int m, p, d, q, l;  // M2L, P2P, deferred, M2P, P2L
};

// Resolves one inherited source S0 for target T.  WRITE = false only counts;
// with WRITE, only the lists whose bit is set in wm are written.
// sel: the target's row of the hybrid selection table, indexed by the source's
// count bucket (nullptr = plain FMM).
enum : unsigned { kWM2L = 1, kWP2P = 2, kWDef = 4, kWM2P = 8, kWP2L = 16 };
template <bool WRITE>
__device__ Counts resolve(const TargetInfo &T, int S0, const CellArrays &c, const ListArrays &L,
                          double theta2, float theta2f, int64_t m_pos, int64_t p_pos, int d_pos,
                          int64_t q_pos, int64_t l_pos, unsigned wm, const uint8_t *__restrict__ sel,
                          uint64_t *hash_keys, int *flags)
{
    Counts n = {0, 0, 0, 0, 0};
    if (S0 & (kP2PFlag | kM2PFlag)) {
        // a P2P or M2P pair chosen at an ancestor of T: record at a leaf, else pass down
        if (!T.leaf) {
            if (WRITE && (wm & kWDef)) L.def_src[d_pos] = S0;
            n.d = 1;
        } else if (S0 & kP2PFlag) {
            if (WRITE && (wm & kWP2P)) {
                L.p2p_src[p_pos] = S0 & kCellMask;
                L.p2p_tgt[p_pos] = T.t;
            }
            n.p = 1;
        } else {
            if (WRITE && (wm & kWM2P)) {
                L.m2p_src[q_pos] = S0 & kCellMask;
                L.m2p_tgt[q_pos] = T.t;
            }
            n.q = 1;
        }
        return n;
    }
    int stk[kStack];
    int sp = 0;
    stk[sp++] = S0;
    while (sp > 0) {
        const int S = stk[--sp];
        const int nchS = c.nchild[S];
        int Cs[3], hs, ls, bs;
        cell_geom(c, S, Cs, hs, ls, bs);
        if (mac_accept(T, Cs, hs, theta2, theta2f)) {
            const int kind = sel ? sel[bs] : 0;  // the target's row of the table, in shared memory
            if (kind == 3) {  // particle-cell: into T's own local expansion, at any level
                if (WRITE && (wm & kWP2L)) {
                    L.p2l_src[l_pos + n.l] = S;
                    L.p2l_tgt[l_pos + n.l] = T.t;
                }
                ++n.l;
            } else if (kind != 0 && !T.leaf) {
                if (WRITE && (wm & kWDef)) L.def_src[d_pos + n.d] = S | (kind == 1 ? kP2PFlag : kM2PFlag);
                ++n.d;
            } else if (kind == 1) {
                if (WRITE && (wm & kWP2P)) {
                    L.p2p_src[p_pos + n.p] = S;
                    L.p2p_tgt[p_pos + n.p] = T.t;
                }
                ++n.p;
            } else if (kind == 2) {
                if (WRITE && (wm & kWM2P)) {
                    L.m2p_src[q_pos + n.q] = S;
                    L.m2p_tgt[q_pos + n.q] = T.t;
                }
                ++n.q;
            } else {
                if (WRITE && (wm & kWM2L)) {
                    L.m2l_src[m_pos + n.m] = S;
                    L.m2l_tgt[m_pos + n.m] = T.t;
                    L.m2l_slot[m_pos + n.m] = hash_insert(hash_keys, class_key(T, ls, Cs, flags), flags);
                }
                ++n.m;
            }
        } else if (T.leaf && nchS == 0) {
            if (WRITE && (wm & kWP2P)) {
                L.p2p_src[p_pos + n.p] = S;
                L.p2p_tgt[p_pos + n.p] = T.t;
            }
            ++n.p;
        } else if (T.leaf || (ls < T.level && nchS > 0)) {
            if (sp + nchS > kStack) {
                atomicOr(&flags[kFlagStack], 1);
                break;
            }
            const int c0 = c.child0[S];
            for (int k = nchS - 1; k >= 0; --k) stk[sp++] = c0 + k;
        } else {
            if (WRITE && (wm & kWDef)) L.def_src[d_pos + n.d] = S;
            ++n.d;
        }
    }
    return n;
}

__device__ __forceinline__ TargetInfo load_target(const CellArrays &c, int t)
{
    TargetInfo T;
    T.t = t;
    T.leaf = c.nchild[t] == 0;
    cell_geom(c, t, T.C, T.h, T.level, T.bt);
    return T;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_excl(int v)
{
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x - v;
}

// Writes the lists of target T whose ni sources F each resolve to one pair:
// ma[r] / mo[r] mark, per round r of 32 sources, the accepted ones (M2L) and the
// others (P2P for a leaf T, deferred otherwise).  The pairs, their order and the
// list offsets are those resolve() would give.
__device__ __forceinline__ void write_single_pairs(const TargetInfo &T, const int *F, int ni, const unsigned *ma,
                                                   const unsigned *mo, const CellArrays &c, const ListArrays &L,
                                                   unsigned long long *__restrict__ counters, int64_t cap_m,
                                                   int64_t cap_p, int64_t cap_d, uint64_t *hash_keys, int *flags)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nr = (ni + 31) >> 5;
    int m = 0, o = 0;
#pragma unroll 1
    for (int r = 0; r < nr; ++r) {
        m += __popc(ma[r]);
        o += __popc(mo[r]);
    }
    const int p = T.leaf ? o : 0, d = T.leaf ? 0 : o;
    unsigned long long om = 0, op = 0, od = 0;
    if (lane == 0) {
        om = atomicAdd(&counters[0], (unsigned long long)m);
        op = atomicAdd(&counters[1], (unsigned long long)p);
        od = atomicAdd(&counters[2], (unsigned long long)d);
    }
    om = __shfl_sync(0xffffffffu, om, 0);
    op = __shfl_sync(0xffffffffu, op, 0);
    od = __shfl_sync(0xffffffffu, od, 0);
    const bool fm = (int64_t)(om + m) <= cap_m, fp = (int64_t)(op + p) <= cap_p, fd = (int64_t)(od + d) <= cap_d;
    const int t = T.t;
    if (lane == 0) {
        L.m2l_off[t] = (int)om;
        L.m2l_cnt[t] = fm ? m : 0;
        L.p2p_off[t] = (int)op;
        L.p2p_cnt[t] = fp ? p : 0;
        L.def_off[t] = (int)od;
        L.def_cnt[t] = fd ? d : 0;
        L.m2p_off[t] = 0;
        L.m2p_cnt[t] = 0;
        L.p2l_off[t] = 0;
        L.p2l_cnt[t] = 0;
    }
    const bool fo = T.leaf ? fp : fd;
    int64_t rm = (int64_t)om, ro = T.leaf ? (int64_t)op : (int64_t)od;
#pragma unroll 1
    for (int r = 0; r < nr; ++r) {
        const int k = r * 32 + lane;
        const unsigned a = ma[r], b = mo[r];
        if (fm && ((a >> lane) & 1u)) {
            const int S = F[k];
            int Cs[3], hs, ls;
            cell_geom(c, S, Cs, hs, ls);
            const int64_t pos = rm + __popc(a & lt);
            L.m2l_src[pos] = S;
            L.m2l_tgt[pos] = t;
            L.m2l_slot[pos] = hash_insert(hash_keys, class_key(T, ls, Cs, flags), flags);
        } else if (fo && ((b >> lane) & 1u)) {
            const int64_t pos = ro + __popc(b & lt);
            if (T.leaf) {
                L.p2p_src[pos] = F[k];
                L.p2p_tgt[pos] = t;
            } else {
                L.def_src[pos] = F[k];
            }
        }
        rm += __popc(a);
        ro += __popc(b);
    }
}

// Writes the lists of target T whose ni sources E each give one pair, of the kind
// recorded as code[k] = -1 - kind: the pairs, their order and the list offsets
// that resolve() would give.
__device__ __forceinline__ void write_kinds(const TargetInfo &T, const int *E, const int *code, int ni,
                                            const CellArrays &c, const ListArrays &L,
                                            unsigned long long *__restrict__ counters, int64_t cap_m, int64_t cap_p,
                                            int64_t cap_d, int64_t cap_q, int64_t cap_l, uint64_t *hash_keys,
                                            int *flags)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    auto list_of = [](int kind) {  // 0 M2L, 1 P2P, 2 deferred, 3 M2P, 4 P2L
        return kind == kOutDefP2P || kind == kOutDefM2P ? 2 : kind;
    };
    int n[5] = {0, 0, 0, 0, 0};
    for (int k0 = 0; k0 < ni; k0 += 32) {
        const int k = k0 + lane;
        const int li = k < ni ? list_of(-1 - code[k]) : -1;
#pragma unroll
        for (int j = 0; j < 5; ++j) n[j] += __popc(__ballot_sync(0xffffffffu, li == j));
    }
    unsigned long long o[5] = {0, 0, 0, 0, 0};
    if (lane == 0) {
        o[0] = atomicAdd(&counters[0], (unsigned long long)n[0]);
        o[1] = atomicAdd(&counters[1], (unsigned long long)n[1]);
        o[2] = atomicAdd(&counters[2], (unsigned long long)n[2]);
        if (n[3]) o[3] = atomicAdd(&counters[3], (unsigned long long)n[3]);
        if (n[4]) o[4] = atomicAdd(&counters[4], (unsigned long long)n[4]);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) o[j] = __shfl_sync(0xffffffffu, o[j], 0);
    const int64_t cap[5] = {cap_m, cap_p, cap_d, cap_q, cap_l};
    bool fit[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) fit[j] = (int64_t)(o[j] + n[j]) <= cap[j];
    const int t = T.t;
    if (lane == 0) {
        L.m2l_off[t] = (int)o[0];
        L.m2l_cnt[t] = fit[0] ? n[0] : 0;
        L.p2p_off[t] = (int)o[1];
        L.p2p_cnt[t] = fit[1] ? n[1] : 0;
        L.def_off[t] = (int)o[2];
        L.def_cnt[t] = fit[2] ? n[2] : 0;
        L.m2p_off[t] = (int)o[3];
        L.m2p_cnt[t] = fit[3] ? n[3] : 0;
        L.p2l_off[t] = (int)o[4];
        L.p2l_cnt[t] = fit[4] ? n[4] : 0;
    }
    int64_t run[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) run[j] = (int64_t)o[j];
    for (int k0 = 0; k0 < ni; k0 += 32) {
        const int k = k0 + lane;
        const int kind = k < ni ? -1 - code[k] : -1;
        const int li = kind >= 0 ? list_of(kind) : -1;
        int64_t pos = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const unsigned m = __ballot_sync(0xffffffffu, li == j);
            if (li == j) pos = run[j] + __popc(m & lt);
            run[j] += __popc(m);
        }
        if (li < 0 || !fit[li]) continue;
        const int S = E[k];
        switch (kind) {
            case kOutM2L: {
                int Cs[3], hs, ls;
                cell_geom(c, S, Cs, hs, ls);
                L.m2l_src[pos] = S;
                L.m2l_tgt[pos] = t;
                L.m2l_slot[pos] = hash_insert(hash_keys, class_key(T, ls, Cs, flags), flags);
                break;
            }
            case kOutP2P:
                L.p2p_src[pos] = S & kCellMask;
                L.p2p_tgt[pos] = t;
                break;
            case kOutM2P:
                L.m2p_src[pos] = S & kCellMask;
                L.m2p_tgt[pos] = t;
                break;
            case kOutP2L:
                L.p2l_src[pos] = S;
                L.p2l_tgt[pos] = t;
                break;
            case kOutDefP2P: L.def_src[pos] = S | kP2PFlag; break;
            case kOutDefM2P: L.def_src[pos] = S | kM2PFlag; break;
            default: L.def_src[pos] = S; break;
        }
    }
}

}  // namespace

// One warp per target of the level [a, b): count the outputs of all inherited
// sources, reserve space for them with one atomic per list, then resolve the
// sources again in the same order and write.  counters[] are running totals over
// the levels; a list whose reservation passes its capacity is not written for the
// target (its count becomes 0) and the host repeats the traversal with larger
// buffers.
__global__ void __launch_bounds__(128, 7)
    k_traverse_level(CellArrays c, ListArrays L, int a, int b, double theta2, float theta2f,
                     const uint8_t *__restrict__ sel, unsigned long long *__restrict__ counters,
                     int64_t cap_m, int64_t cap_p, int64_t cap_d, int64_t cap_q, int64_t cap_l,
                     uint64_t *__restrict__ hash_keys, int *__restrict__ flags, const int *__restrict__ sz,
                     int level)
{
    __shared__ int sF[4][2][kFrontier];
    __shared__ int sN[4][kFrontier];  // per source of the frontier: its children when split, else -1
    __shared__ int sCnt[4][5][kCountCache];  // per-source counts of the count pass (first kCountCache)
    __shared__ uint8_t sRow[4][kSelNB];      // the target's row of the selection table
    __shared__ unsigned sMa[4][kFrontier / 32], sMo[4][kFrontier / 32];  // a round's accepted / single-pair masks
    if (sz) {
        a = sz[kSzLevel + level];
        b = sz[kSzLevel + level + 1];
    }
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int t = a + warp;
    if (t >= b) return;
    const TargetInfo T = load_target(c, t);
    const uint8_t *row = nullptr;  // the target's row of the selection table
    if (sel) {
        for (int k = lane; k < kSelNB; k += 32) sRow[wib][k] = sel[T.bt * kSelNB + k];
        __syncwarp();
        row = sRow[wib];
    }
    const int P = c.parent[t];
    const int i0 = L.def_off[P];
    int ni = L.def_cnt[P];
    const int *F = L.def_src + i0;
    if (ni <= kFrontier) {
        // A target resolves every inherited source it does not accept by a
        // depth-first walk of the source's subtree, one source per lane; next to a
        // dense region a few sources carry almost all the work.  Instead, rounds of
        // the whole warp classify every source once (accepted; split, when it is
        // not accepted, has children and the target is a leaf or smaller than it;
        // or neither) and replace the split ones by their children while the list
        // fits in kFrontier entries.  The set of pairs does not change, only the
        // order of discovery.  When a round splits nothing and every source gives
        // exactly one pair (no selection table), the pairs are placed by ballot and
        // no walk is needed.
        int cur = 0;
        for (int k = lane; k < ni; k += 32) sF[wib][0][k] = F[k];
        __syncwarp();
        for (int round = 0; round < 8; ++round) {
            const int *E = sF[wib][cur];
            int *nsplit = sN[wib];  // per source: its children when split, else -1
            unsigned *ma = sMa[wib], *mo = sMo[wib];
            int total = 0;
            bool any_split = false, single = true;
            bool plain = true;  // every pair of the round is of the kind the plain FMM gives it
            const int nr = (ni + 31) >> 5;
            // a rolled loop: unrolled over the kFrontier / 32 rows, the classification
            // and pair writing make a code footprint that stalls on instruction fetch
#pragma unroll 1
            for (int r = 0; r < nr; ++r) {
                {
                    const int k = r * 32 + lane;
                    bool acc = false, sp = false, one = false, pk = true;
                    int nc = 0;
                    if (k < ni) {
                        const int S = E[k];
                        nc = 1;
                        int kind = kOutDef;  // the source's single pair when it is not split
                        pk = !(S & (kP2PFlag | kM2PFlag));
                        if (pk) {
                            int Cs[3], hs, ls, bs;
                            cell_geom(c, S, Cs, hs, ls, bs);
                            const int nch = c.nchild[S];
                            acc = mac_accept(T, Cs, hs, theta2, theta2f);
                            sp = !acc && nch > 0 && (T.leaf || ls < T.level);
                            one = !sp;
                            if (sp) nc = nch;
                            if (acc) {
                                const int kd = sel ? row[bs] : 0;  // as resolve()
                                pk = kd == 0;
                                kind = kd == 3 ? kOutP2L
                                       : kd != 0 && !T.leaf ? (kd == 1 ? kOutDefP2P : kOutDefM2P)
                                       : kd == 1 ? kOutP2P
                                       : kd == 2 ? kOutM2P
                                                 : kOutM2L;
                            } else if (T.leaf) {
                                kind = kOutP2P;  // (a leaf source; others are split)
                            }
                        } else if (T.leaf) {
                            kind = (S & kP2PFlag) ? kOutP2P : kOutM2P;  // a pair chosen at an ancestor
                        }
                        nsplit[k] = sp ? nc : -1 - kind;
                    }
                    const unsigned ba = __ballot_sync(0xffffffffu, acc), bo = __ballot_sync(0xffffffffu, one && !acc);
                    if (lane == 0) {
                        ma[r] = ba;
                        mo[r] = bo;
                    }
                    single = __all_sync(0xffffffffu, k >= ni || one) && single;
                    plain = __all_sync(0xffffffffu, pk) && plain;
                    any_split = __any_sync(0xffffffffu, sp) || any_split;
                    total += warp_sum(nc);
                }
            }
            if (!any_split) {
                if (single && (!sel || plain)) {
                    // (with a selection table whose entries for these pairs are all M2L,
                    // the lists are those of the plain FMM)
                    __syncwarp();
                    write_single_pairs(T, E, ni, ma, mo, c, L, counters, cap_m, cap_p, cap_d, hash_keys, flags);
                    return;
                }
                if (sel) {  // with a selection table every source left gives one pair of its recorded kind
                    __syncwarp();
                    write_kinds(T, E, nsplit, ni, c, L, counters, cap_m, cap_p, cap_d, cap_q, cap_l, hash_keys,
                                flags);
                    return;
                }
                break;
            }
            if (total > kFrontier) break;
            __syncwarp();
            int base = 0;
            for (int k0 = 0; k0 < ni; k0 += 32) {
                const int k = k0 + lane;
                const int ns = k < ni ? nsplit[k] : 0;
                const int nc = k < ni ? (ns > 0 ? ns : 1) : 0;
                const int pos = base + warp_excl(nc);
                if (k < ni) {
                    const int S = E[k];
                    int *dst = sF[wib][cur ^ 1] + pos;
                    if (ns > 0) {
                        const int c0 = c.child0[S];
                        for (int j = 0; j < ns; ++j) dst[j] = c0 + j;
                    } else {
                        dst[0] = S;
                    }
                }
                base += warp_sum(nc);
            }
            __syncwarp();
            cur ^= 1;
            ni = total;
        }
        __syncwarp();
        F = sF[wib][cur];
    }
    int m = 0, p = 0, d = 0, q = 0, l = 0;
    for (int k = lane; k < ni; k += 32) {
        const Counts n = resolve<false>(T, F[k], c, L, theta2, theta2f, 0, 0, 0, 0, 0, 0u, row, nullptr, flags);
        if (k < kCountCache) {
            sCnt[wib][0][k] = n.m;
            sCnt[wib][1][k] = n.p;
            sCnt[wib][2][k] = n.d;
            sCnt[wib][3][k] = n.q;
            sCnt[wib][4][k] = n.l;
        }
        m += n.m;
        p += n.p;
        d += n.d;
        q += n.q;
        l += n.l;
    }
    m = warp_sum(m);
    p = warp_sum(p);
    d = warp_sum(d);
    q = warp_sum(q);
    l = warp_sum(l);
    unsigned long long om = 0, op = 0, od = 0, oq = 0, ol = 0;
    if (lane == 0) {
        om = atomicAdd(&counters[0], (unsigned long long)m);
        op = atomicAdd(&counters[1], (unsigned long long)p);
        od = atomicAdd(&counters[2], (unsigned long long)d);
        if (q) oq = atomicAdd(&counters[3], (unsigned long long)q);
        if (l) ol = atomicAdd(&counters[4], (unsigned long long)l);
    }
    om = __shfl_sync(0xffffffffu, om, 0);
    op = __shfl_sync(0xffffffffu, op, 0);
    od = __shfl_sync(0xffffffffu, od, 0);
    oq = __shfl_sync(0xffffffffu, oq, 0);
    ol = __shfl_sync(0xffffffffu, ol, 0);
    // Each list is written only where it fits.  The deferred list is what the next
    // level reads, so while it fits the traversal goes on and every count stays
    // exact: one regrow of the lists that overflowed then suffices.
    const bool fm = (int64_t)(om + m) <= cap_m, fp = (int64_t)(op + p) <= cap_p, fd = (int64_t)(od + d) <= cap_d,
               fq = (int64_t)(oq + q) <= cap_q, fl = (int64_t)(ol + l) <= cap_l;
    const unsigned wm = (fm ? kWM2L : 0u) | (fp ? kWP2P : 0u) | (fd ? kWDef : 0u) | (fq ? kWM2P : 0u) | (fl ? kWP2L : 0u);
    if (lane == 0) {
        L.m2l_off[t] = (int)om;
        L.m2l_cnt[t] = fm ? m : 0;
        L.p2p_off[t] = (int)op;
        L.p2p_cnt[t] = fp ? p : 0;
        L.def_off[t] = (int)od;
        L.def_cnt[t] = fd ? d : 0;
        L.m2p_off[t] = (int)oq;
        L.m2p_cnt[t] = fq ? q : 0;
        L.p2l_off[t] = (int)ol;
        L.p2l_cnt[t] = fl ? l : 0;
    }
    if (!wm) return;
    int64_t rm = 0, rp = 0, rq = 0, rl = 0;
    int rd = 0;
    for (int k0 = 0; k0 < ni; k0 += 32) {
        const int k = k0 + lane;
        const int S0 = k < ni ? F[k] : -1;
        Counts n = {0, 0, 0, 0, 0};
        if (S0 >= 0 && k < kCountCache)  // counted by this lane in the count pass
            n = {sCnt[wib][0][k], sCnt[wib][1][k], sCnt[wib][2][k], sCnt[wib][3][k], sCnt[wib][4][k]};
        else if (S0 >= 0)
            n = resolve<false>(T, S0, c, L, theta2, theta2f, 0, 0, 0, 0, 0, 0u, row, nullptr, flags);
        const int em = warp_excl(n.m), ep = warp_excl(n.p), ed = warp_excl(n.d), eq = warp_excl(n.q),
                  el = warp_excl(n.l);
        if (S0 >= 0)
            resolve<true>(T, S0, c, L, theta2, theta2f, (int64_t)om + rm + em, (int64_t)op + rp + ep,
                          (int)od + rd + ed, (int64_t)oq + rq + eq, (int64_t)ol + rl + el, wm, row, hash_keys,
                          flags);
        rm += warp_sum(n.m);
        rp += warp_sum(n.p);
        rd += warp_sum(n.d);
        rq += warp_sum(n.q);
        rl += warp_sum(n.l);
    }
}

// ---------------------------------------------------------------- classes

__global__ void k_hash_flags(const uint64_t *__restrict__ hash_keys, int *__restrict__ flag)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHashCap) flag[i] = hash_keys[i] != kHashEmpty;
}

__global__ void k_hash_compact(const uint64_t *__restrict__ hash_keys, const int *__restrict__ ex,
                               uint64_t *__restrict__ ukeys, uint32_t *__restrict__ uslot)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHashCap && hash_keys[i] != kHashEmpty) {
        ukeys[ex[i]] = hash_keys[i];
        uslot[ex[i]] = i;
    }
}

// Level 0 of the traversal, one pair (root, root) per system: a root that is a
// leaf gets the P2P pair (root, root), any other root defers itself to its
// children.  One block, deterministic compaction (block-wide scans in chunks);
// counters[] receive the list sizes.
__global__ void k_root_lists(CellArrays c, ListArrays L, int nsys, unsigned long long *counters)
{
    __shared__ int sw[64];
    int base_p = 0, base_d = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool valid = s < nsys;
        const bool leaf = valid && c.nchild[s] == 0;
        const bool defer = valid && !leaf;
        const unsigned bp = __ballot_sync(0xffffffffu, leaf), bd = __ballot_sync(0xffffffffu, defer);
        if (lane == 0) {
            sw[warp] = __popc(bp);
            sw[32 + warp] = __popc(bd);
        }
        __syncthreads();
        int op = 0, od = 0, tp = 0, td = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) {
                op += sw[w];
                od += sw[32 + w];
            }
            tp += sw[w];
            td += sw[32 + w];
        }
        const unsigned lt = (1u << lane) - 1u;
        op += base_p + __popc(bp & lt);
        od += base_d + __popc(bd & lt);
        if (valid) {
            L.m2l_off[s] = 0;
            L.m2l_cnt[s] = 0;
            L.p2p_off[s] = op;
            L.p2p_cnt[s] = leaf ? 1 : 0;
            L.def_off[s] = od;
            L.def_cnt[s] = leaf ? 0 : 1;
            L.m2p_off[s] = 0;
            L.m2p_cnt[s] = 0;
            L.p2l_off[s] = 0;
            L.p2l_cnt[s] = 0;
            if (leaf) {
                L.p2p_src[op] = s;
                L.p2p_tgt[op] = s;
            } else {
                L.def_src[od] = s;
            }
        }
        base_p += tp;
        base_d += td;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counters[0] = 0;
        counters[1] = (unsigned long long)base_p;
        counters[2] = (unsigned long long)base_d;
        counters[3] = 0;
        counters[4] = 0;
    }
}

// Sorts up to a few thousand distinct keys: the rank of a key is the number of
// smaller keys (one thread per key).  slot_class[slot of the key] = its rank.
__global__ void __launch_bounds__(128)
    k_rank_classes(const uint64_t *__restrict__ ukeys, const uint32_t *__restrict__ uslot, int n,
                   uint64_t *__restrict__ sorted_keys, int *__restrict__ slot_class, const int *__restrict__ sz)
{
    if (sz) n = sz[kSzClasses];
    // each block ranks 128 keys against all n, staged through shared memory
    __shared__ uint64_t sk[2048];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t k = i < n ? ukeys[i] : 0;
    int r = 0;
    for (int j0 = 0; j0 < n; j0 += 2048) {
        const int m = min(2048, n - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) sk[j] = ukeys[j0 + j];
        __syncthreads();
        for (int j = 0; j < m; ++j) r += sk[j] < k;
    }
    if (i < n) {
        sorted_keys[r] = k;
        slot_class[uslot[i]] = r;
    }
}

__global__ void k_slot_to_class(const uint32_t *__restrict__ uslot, int nclass,
                                int *__restrict__ slot_class)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nclass) slot_class[uslot[r]] = r;
}

__global__ void k_m2l_class(uint32_t *__restrict__ m2l_slot, int64_t n,
                            const int *__restrict__ slot_class, const unsigned long long *__restrict__ dn)
{
    if (dn) n = (int64_t)*dn;
    // four elements per thread and round, their loads issued together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint32_t sl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sl[u] = i0 + u * stride < n ? m2l_slot[i0 + u * stride] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * stride < n) m2l_slot[i0 + u * stride] = (uint32_t)slot_class[sl[u]];
    }
}

// ---------------------------------------------------------------- tiles

__global__ void k_tile_bitmap(const int *__restrict__ m2l_tgt, const uint32_t *__restrict__ m2l_class,
                              int64_t n, const int *__restrict__ cell_tile, int nwords,
                              uint32_t *__restrict__ bitmap, const unsigned long long *__restrict__ dn)
{
    if (dn) n = (int64_t)*dn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cl = m2l_class[i];
        const int tile = cell_tile[m2l_tgt[i]];
        uint32_t *w = &bitmap[(int64_t)tile * nwords + (cl >> 5)];
        const uint32_t bit = 1u << (cl & 31);
        if (!(__ldg(w) & bit)) atomicOr(w, bit);
    }
}

__global__ void k_tile_popc(const uint32_t *__restrict__ bitmap, int ntiles, int nwords,
                            int *__restrict__ cnt)
{
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    int s = 0;
    for (int w = lane; w < nwords; w += 32) s += __popc(bitmap[(int64_t)tile * nwords + w]);
    s = warp_sum(s);
    if (lane == 0) cnt[tile] = s;
}

// One warp per tile: word prefix counts and the list of (cache slot of) classes.
__global__ void k_tile_entries(const uint32_t *__restrict__ bitmap, int ntiles, int nwords,
                               const int *__restrict__ entry_base, int *__restrict__ word_prefix,
                               int *__restrict__ entry_class, const int *__restrict__ class_slot, int entry_cap)
{
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    int run = entry_base[tile];
    for (int w0 = 0; w0 < nwords; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t bits = w < nwords ? bitmap[(int64_t)tile * nwords + w] : 0u;
        const int pc = __popc(bits);
        const int ex = warp_excl(pc);
        if (w < nwords) {
            word_prefix[(int64_t)tile * nwords + w] = run + ex;
            uint32_t rem = bits;
            int e = run + ex;
            while (rem) {
                const int bpos = __ffs(rem) - 1;
                rem &= rem - 1;
                if (e < entry_cap) entry_class[e] = class_slot[w * 32 + bpos];
                ++e;
            }
        }
        run += warp_sum(pc);
    }
}

// The gather index of every M2L pair, src[entry * kTile + row], written row by
// row in tile order: warp w takes row w % kTile of tile w / kTile, and its lanes
// take 32 of the row's pairs at a time (the cell's pairs are contiguous).  Warps start in order, so the rows in flight belong to a few
// dozen tiles, whose entries (a few hundred kilobytes each) stay in the L2
// cache while their writes merge; in pair order the writes spread over the
// whole array (a quarter of a gigabyte at 4M Plummer points), where each 4-byte
// write costs a partial sector in DRAM.
__global__ void __launch_bounds__(128)
    k_tile_src_rows(const int *__restrict__ tile_cells, int ntiles, const int *__restrict__ m2l_off,
                    const int *__restrict__ m2l_cnt, const int *__restrict__ m2l_src,
                    const uint32_t *__restrict__ m2l_class, int nwords, const uint32_t *__restrict__ bitmap,
                    const int *__restrict__ word_prefix, int *__restrict__ src, const int *__restrict__ sz,
                    int entry_cap)
{
    if (sz) {
        if (sz[kSzAbort]) return;  // (class ids may be unconverted hash slots)
        ntiles = sz[kSzTiles];
    }
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)ntiles * kTile) return;
    const int tile = (int)(gw / kTile), r = (int)(gw % kTile);
    const int cell = tile_cells[gw];
    if (cell < 0) return;
    const int o = m2l_off[cell], cnt = m2l_cnt[cell];
    const uint32_t *bm = bitmap + (int64_t)tile * nwords;
    const int *wp = word_prefix + (int64_t)tile * nwords;
    for (int k = lane; k < cnt; k += 32) {
        const uint32_t cl = m2l_class[o + k];
        const int s = m2l_src[o + k];
        if ((int)(cl >> 5) >= nwords) continue;
        const uint32_t below = bm[cl >> 5] & ((1u << (cl & 31)) - 1u);
        const int e = wp[cl >> 5] + __popc(below);
        if (e < entry_cap) src[(int64_t)e * kTile + r] = s;
    }
}

// ---------------------------------------------------------------- replayed plans

__global__ void k_check_lists(const unsigned long long *__restrict__ counters, int64_t cap_m, int64_t cap_p,
                              int64_t cap_d, int64_t cap_q, int64_t cap_l, unsigned long long *__restrict__ totals,
                              int *__restrict__ sz)
{
    const int64_t cap[5] = {cap_m, cap_p, cap_d, cap_q, cap_l};
    bool fits = true;
    for (int k = 0; k < 5; ++k) fits = fits && (int64_t)counters[k] <= cap[k];
    if (!fits) sz[kSzAbort] = 1;
    for (int k = 0; k < 5; ++k) totals[k] = fits ? counters[k] : 0ull;
}

__global__ void k_plan_classes(const int *__restrict__ nclass_dev, int nclass_cap, int *__restrict__ sz,
                               unsigned long long *__restrict__ totals)
{
    const int n = *nclass_dev;
    if (n > nclass_cap) {
        sz[kSzAbort] = 1;
        sz[kSzClasses] = 0;
        totals[0] = 0ull;  // no class ids: no M2L pair is placed
    } else {
        sz[kSzClasses] = n;
    }
}

__global__ void k_class_lookup(const uint64_t *__restrict__ sorted_keys, const int *__restrict__ sz,
                               const uint64_t *__restrict__ hkeys, const int *__restrict__ hslots, uint32_t hcap,
                               int *__restrict__ class_slot, int *__restrict__ szw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sz[kSzClasses]) return;
    const uint64_t k = sorted_keys[i];
    uint32_t h = (uint32_t)((k * 0x9e3779b97f4a7c15ull) >> 40) & (hcap - 1);
    int slot = -1;
    for (uint32_t probe = 0; probe < hcap; ++probe, h = (h + 1) & (hcap - 1)) {
        const uint64_t hk = hkeys[h];
        if (hk == k) {
            slot = hslots[h];
            break;
        }
        if (hk == kHashEmpty) break;
    }
    if (slot < 0) {  // a class the plan has no operator for
        szw[kSzAbort] = 1;
        slot = 0;
    }
    class_slot[i] = slot;
}

// One block: every thread reads the total before any thread clears it.
__global__ void k_check_entries(int *__restrict__ entry_base, int ntiles_cap, int nent_cap, int *__restrict__ sz)
{
    const int n = entry_base[ntiles_cap];
    __syncthreads();
    if (n <= nent_cap) {
        if (threadIdx.x == 0) sz[kSzEntries] = n;
        return;
    }
    if (threadIdx.x == 0) {
        sz[kSzAbort] = 1;
        sz[kSzEntries] = 0;
    }
    for (int t = threadIdx.x; t <= ntiles_cap; t += blockDim.x) entry_base[t] = 0;  // every tile empty
}

}  // namespace fmm
