/*
 * fmm.h -- C ABI of the GB300 fast multipole library for the 3-D Laplace
 * potential and gradient (Yokota & Barba, "Hierarchical N-body simulations with
 * auto-tuning for heterogeneous systems").
 *
 * The problem (Results section: "Laplace kernel potential and force", targets
 * equal to sources): for N charges q_j at x_j,
 *     phi_i  = sum_{j, r_ij > 0} q_j / r_ij
 *     grad_i = -sum_{j, r_ij > 0} q_j (x_i - x_j) / r_ij^3      (grad_i = del phi(x_i))
 * The paper's force on particle i is -q_i grad_i.  Pairs at zero distance
 * (including i = j) contribute nothing.
 *
 * The method (sections "Hybrid treecode/FMM algorithm" and "Dual tree
 * traversal"): an adaptive octree with at most ncrit particles per leaf, a
 * stack-based dual tree traversal with the multipole acceptance criterion
 * theta = (r_t + r_s)/R, spherical-harmonic expansions of order p with
 * cell-cell (M2L) far-field and particle-particle (P2P) near-field
 * interactions, plus the P2M/M2M upward and L2L/L2P downward passes.
 *
 * Conventions for every entry point:
 *   * Coordinates are float32, row-major [N][3] (x, y, z interleaved); charges
 *     float32 [N]; phi float32 [N]; grad float32 [N][3].  Outputs are in the
 *     caller's particle order.  Inputs are never modified.
 *   * Pointers are DEVICE pointers of the current CUDA device unless the name
 *     says _host.  The caller owns all buffers; the library keeps no pointer
 *     after returning.
 *   * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  The plain path synchronises `stream` where it must read sizes
 *     back (once per tree level); on return the outputs are complete.
 *   * Internal scratch comes from a library-owned pool per device, grown on
 *     demand and kept until process exit.  Calls on one device are serialised
 *     by a lock; calls on different devices may run concurrently.
 *   * On any status other than FMM_OK the outputs are unspecified and
 *     fmm_last_error() describes the failure.  Invalid arguments are detected
 *     before any device work is enqueued.
 */
#ifndef GB300_FMM_H
#define GB300_FMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = 1,       /* an argument is out of range or a pointer is NULL */
    FMM_ERR_NONFINITE = 2, /* a coordinate is NaN or infinite (found while bounding the box) */
    FMM_ERR_CAPACITY = 3,  /* an interaction list outgrew its bound after one regrow */
    FMM_ERR_CUDA = 4,      /* a CUDA call failed; fmm_last_error() has the message */
    FMM_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    FMM_ERR_NOMEM = 6      /* device or pinned host memory could not be allocated */
} fmm_status;

/* Arithmetic of the M2L translations (the other steps are fixed: FP32
 * particle/expansion arithmetic, FP64 box quantisation and operator tables). */
enum {
    FMM_PREC_FP32 = 0,   /* FP32 FMA on the CUDA cores */
    FMM_PREC_TF32X3 = 1, /* tensor cores, operands split hi+lo in TF32, FP32 accumulate */
    FMM_PREC_BF16X3 = 2  /* tensor cores, operands split hi+lo in BF16, FP32 accumulate */
};

/* Interaction type of the pairs the MAC accepts (section "A new hybrid
 * treecode-FMM with auto-tuning": the type is chosen during the traversal to
 * minimise the cost, and particle-particle interactions may be taken above the
 * leaf level).  Every mode is exact in the sense that a pair not taken as M2L is
 * taken as P2P, so the far-field error can only shrink.
 * The choice is a table sel[b(n_t) * FMM_SELECT_NB + b(n_s)] (0 = M2L, 1 = P2P,
 * 2 = M2P: the source multipole evaluated at every target particle, the treecode's
 * cell-particle interaction; 3 = P2L: the source particles added straight into the
 * target cell's local expansion)
 * over the particle counts n_t, n_s of the target and source cells, with the
 * count bucket b(n) = n - 1 for n < 4, else 3 + 4(e - 2) + ((n >> (e - 2)) & 3),
 * e = floor(log2 n) (four buckets per octave). */
enum {
    FMM_SELECT_PLAIN = 0,    /* M2L for every accepted pair: the plain FMM */
    FMM_SELECT_AUTOTUNE = 1, /* table from kernels timed on artificial cells (kernel
                                pre-calculation), measured once per device, p and precision */
    FMM_SELECT_LEARNED = 2,  /* table from the learned cost model (fmm_cost_model_*) */
    FMM_SELECT_TABLE = 3,    /* the caller's table in fmm_options.select_table */
    FMM_SELECT_TREECODE = 4  /* M2P for every accepted pair: the paper's treecode (Results
                                section), on the same tree and traversal */
};
#define FMM_SELECT_NB 128

typedef struct {
    int max_depth;      /* deepest tree level, 1..21 (0 selects 21) */
    int precision_mode; /* FMM_PREC_* */
    int select_mode;    /* FMM_SELECT_* */
    int deterministic;  /* 1 = bitwise-reproducible results (the only mode implemented) */
    /* FMM_SELECT_TABLE: HOST uint8[FMM_SELECT_NB][FMM_SELECT_NB], read during the
     * call only; ignored by the other modes. */
    const unsigned char *select_table;
    /* tensor-core M2L schedule: (target tile, offset class) blocks per work unit,
     * 0 = automatic (about six units per SM, at least 8 blocks) */
    int m2l_unit_blocks;
    /* 0 (default): the far-field chain (offset classes, tiles, M2L, L2L, L2P) runs
     * on its own stream beside P2P and takes SMs as P2P's blocks retire; 1: it
     * waits until P2P has finished, so that each phase's time in fmm_stats is
     * that phase alone (slower; for measurements).  Plans ignore it. */
    int serialize_phases;
    /* 1 (default): a solve without statistics and without serialize_phases whose
     * key -- N, the system offsets, p, theta, ncrit, max_depth, precision_mode,
     * select_mode, m2l_unit_blocks and the selection table's content -- equals
     * the previous such call's on this device captures a plan after it solves
     * (as fmm_plan_create, capacities 1.25x this solve's), and later calls with
     * that key replay it: every step of the solve still runs, in one graph
     * launch with every size on the device, reading this call's xyz and q and
     * writing its phi and grad in place (any arrays: their addresses are handed
     * to the plan at each replay), and the results are bit-identical to a plain
     * solve.  A replay that outgrows the plan is solved
     * again plainly and the plan is dropped.  The plan's memory stays allocated
     * until a call with another key captures its own.  The first two calls with
     * a key are plain solves; the second also captures.  0: always a plain
     * solve. */
    int replay;
} fmm_options;

typedef struct {
    int64_t ncells, nleaves, depth;
    int64_t n_p2p_pairs, n_p2p_interactions; /* leaf pairs; sum over pairs of n_t * n_s */
    int64_t n_m2l_pairs, n_offset_classes;   /* cell pairs; distinct translation offsets */
    int64_t n_m2l_blocks;                    /* (target tile, offset class) GEMM blocks */
    int64_t n_launches;                      /* kernels this library launched for the solve */
    /* per-phase device time in ms (measured with events when stats are requested):
     * ms_tree keys, sort and tree; ms_traverse the dual-tree traversal; ms_upward
     * P2M and M2M; ms_m2l the M2L kernel and its unit reduction; ms_downward L2L
     * and L2P; ms_p2p the P2P kernel, which runs beside the far-field chain (the
     * offset classes and tiles are built on the far-field stream while P2P runs
     * and are in no phase; unless fmm_options.serialize_phases is set, P2P and
     * the far-field phases share the GPU and their times overlap); ms_total the
     * whole solve */
    float ms_tree, ms_upward, ms_traverse, ms_m2l, ms_downward, ms_p2p, ms_total;
    int64_t n_m2p_pairs; /* (target leaf, source cell) cell-particle pairs */
    int64_t n_p2l_pairs; /* (target cell, source cell) particle-cell pairs */
} fmm_stats;

/* Fills *opt with the defaults (max_depth 21, FP32 M2L, plain FMM, deterministic,
 * phases overlapped, repeated solves replayed). */
void fmm_default_options(fmm_options *opt);

/* The FMM solve.  Arguments must satisfy N >= 1, 1 <= p <= 20, 0 < theta < 1,
 * ncrit >= 1 and N < 2^31; otherwise FMM_ERR_ARG.  p is the expansion order
 * (section "Hybrid treecode/FMM algorithm"), theta the MAC (Results section),
 * ncrit the maximum number of particles per leaf (Results section). */
fmm_status fmm_laplace3d(const float *xyz, const float *q, int64_t N, int p, double theta,
                         int ncrit, float *phi, float *grad, void *stream);

/* As fmm_laplace3d with options (NULL = defaults) and optional statistics
 * (NULL = none; non-NULL adds event timing and one extra synchronisation). */
fmm_status fmm_laplace3d_ex(const float *xyz, const float *q, int64_t N, int p, double theta,
                            int ncrit, float *phi, float *grad, void *stream,
                            const fmm_options *opt, fmm_stats *stats);

/* As fmm_laplace3d_ex but every array is in HOST memory (pageable or pinned):
 * the library copies the inputs to the device, solves on `stream` and copies
 * the results back before returning. */
fmm_status fmm_laplace3d_host(const float *xyz_host, const float *q_host, int64_t N, int p,
                              double theta, int ncrit, float *phi_host, float *grad_host,
                              void *stream, const fmm_options *opt, fmm_stats *stats);

/* Many independent systems in one solve.  System s is the particles
 * [offsets[s], offsets[s+1]) of xyz/q/phi/grad; offsets is a HOST array of
 * nsys + 1 increasing values with offsets[0] = 0 and at least one particle per
 * system (else FMM_ERR_ARG).  Each system gets its own bounding box and tree
 * (one root per system, all trees built, traversed and evaluated together by
 * the same kernel launches); no interaction crosses systems.  Every system uses
 * the same p, theta, ncrit and options.  Same pointer conventions as
 * fmm_laplace3d_ex; FMM_EXPORT_BOX then returns double[nsys][4]. */
fmm_status fmm_laplace3d_batched(const float *xyz, const float *q, const int64_t *offsets,
                                 int nsys, int p, double theta, int ncrit, float *phi, float *grad,
                                 void *stream, const fmm_options *opt, fmm_stats *stats);

/* Exact all-pairs sum on the GPU (the O(N^2) direct summation of the paper's
 * Introduction): FP32 arithmetic, same conventions as fmm_laplace3d. */
fmm_status fmm_direct(const float *xyz, const float *q, int64_t N, float *phi, float *grad,
                      void *stream);

/* Failure-detection self-test (the paper has no counterpart).  Runs one kernel
 * whose bounded wait can never be satisfied (an mbarrier nothing arrives at),
 * with `polls` polls (1..2^26) before it gives up, exactly as the M2L pipeline's
 * waits do.  The expected result is FMM_ERR_TIMEOUT, read from the device flag;
 * the context stays usable.  `stream` as for the solves. */
fmm_status fmm_selftest_wait_timeout(int64_t polls, void *stream);

/* Copies an intermediate array of the most recent successful solve on the
 * current device into host memory `dst` of `capacity` bytes; *needed (may be
 * NULL) receives the byte size.  Returns FMM_ERR_ARG if no solve has run or
 * capacity is too small.  Cells are in the library's order (level by level,
 * Morton order within a level); cell-index arrays refer to that order.
 *   FMM_EXPORT_BOX        double[nsys][4]: lo_x, lo_y, lo_z, side of each system's box
 *   FMM_EXPORT_KEYS       uint64[N] Morton keys in sorted order
 *   FMM_EXPORT_ORDER      int32[N]  original index of each sorted position
 *   FMM_EXPORT_CELLS      int64[ncells][6]: level, key prefix, begin, end, parent, nchild
 *   FMM_EXPORT_P2P        int32[n][2]: target leaf, source cell (a leaf in the plain
 *                         FMM; with a selection table a P2P pair chosen above the
 *                         leaf level appears once per target leaf below it)
 *   FMM_EXPORT_M2L        int32[n][3]: target cell, source cell, offset class
 *   FMM_EXPORT_MULTIPOLE  float[ncells][P2pad] unit-scaled multipoles (see below)
 *   FMM_EXPORT_LOCAL      float[ncells][P2pad] unit-scaled local expansions
 *   FMM_EXPORT_SELECT     uint8[FMM_SELECT_NB][FMM_SELECT_NB] selection table the
 *                         solve used (all zero for the plain FMM)
 *   FMM_EXPORT_M2P        int32[n][2]: target leaf, source cell of the cell-particle
 *                         pairs (a pair chosen above the leaf level appears once per
 *                         target leaf below it)
 *   FMM_EXPORT_P2L        int32[n][2]: target cell, source cell of the particle-cell pairs
 * Expansion rows hold, for n = 0..p, Re c_n^0 then (Re c_n^m, Im c_n^m) for
 * m = 1..n ((p+1)^2 values, zero-padded to P2pad = a multiple of 32), scaled
 * by s^-n (multipoles) or s^(n+1) (locals) with s the cell side. */
enum {
    FMM_EXPORT_BOX = 0,
    FMM_EXPORT_KEYS = 1,
    FMM_EXPORT_ORDER = 2,
    FMM_EXPORT_CELLS = 3,
    FMM_EXPORT_P2P = 4,
    FMM_EXPORT_M2L = 5,
    FMM_EXPORT_MULTIPOLE = 6,
    FMM_EXPORT_LOCAL = 7,
    FMM_EXPORT_SELECT = 8,
    FMM_EXPORT_M2P = 9,
    FMM_EXPORT_P2L = 10
};
fmm_status fmm_export(int what, void *dst, int64_t capacity, int64_t *needed);

/* ------------------------------------------------------------------------
 * Hybrid selection: pre-timed kernels and the learned cost model
 * ------------------------------------------------------------------------
 * Section "Kernel pre-calculation": the interaction kernels are timed on
 * artificial coordinates and charges, and the traversal selects the cheapest
 * interaction type from those timings.  FMM_SELECT_AUTOTUNE does exactly that:
 * the P2P kernel is timed on artificial leaves over a grid of target and source
 * counts (1..512, launches sized like real solves), the M2L time per pair comes
 * from plain solves of an artificial uniform cube (2^18 particles) at the
 * solve's p, theta and precision, and a pair becomes P2P where the (log-log
 * interpolated) P2P time is below the M2L time.  Measured once per device and
 * cached.
 * FMM_SELECT_LEARNED replaces the interpolation by a network (3 layers, hidden
 * width 64, FP16 parameters) trained on the GPU on those timings:
 *   x = (log2 n_t, log2 n_s, sep, p), sep = R / (r_t + r_s) (1/theta for the
 *   table), y = (ln ns per P2P pair, ln ns per M2L pair);
 *   u = (x - (5, 5, 3, 8)) / (4, 4, 1.5, 4), h1 = tanh(W1 u + b1),
 *   h2 = tanh(W2 h1 + b2), y = W3 h2 + b3;
 *   parameters in the order W1 (64x4 row-major), b1, W2 (64x64), b2, W3 (2x64), b3;
 *   loss = sum m (y - t)^2 / sum m over the masked outputs; Adam (lr 3e-3,
 *   betas 0.9/0.999, eps 1e-8) on FP32 master weights, FP16 copy for the forward.
 * The table takes, for each bucket, the geometric mean of its count range.
 * Until a model is trained or set, FMM_SELECT_LEARNED uses the pre-timed table. */
#define FMM_COST_MODEL_PARAMS 4610

typedef struct {
    int64_t n_samples_p2p, n_samples_m2l; /* training samples of each kind */
    int steps;                            /* Adam steps (full batch) */
    float loss_initial, loss_final;       /* loss before the first and after the last step */
    float agreement;                      /* worst fraction, over the training (p, theta) grid, of
                                             table entries with counts <= 4096 where the learned
                                             table equals the pre-timed one */
    float ms_pretime, ms_train;           /* time to generate the samples / to train */
} fmm_cost_model_info;

/* The selection table FMM_SELECT_AUTOTUNE or FMM_SELECT_LEARNED would use for
 * (p, theta, precision) on the current device (measuring it if needed):
 * host uint8[FMM_SELECT_NB][FMM_SELECT_NB]. */
fmm_status fmm_selection_table(int select_mode, int p, double theta, int precision_mode,
                               unsigned char *table);
/* Generates timing samples (P2P on artificial leaves; M2L from artificial solves
 * at p = p_lo..p_hi and theta in {0.35, 0.45, 0.55, 0.65}, in the given M2L
 * precision), initialises the network from `seed` and trains it for `steps`
 * full-batch Adam steps on the GPU.  info may be NULL. */
fmm_status fmm_cost_model_train(int precision_mode, int p_lo, int p_hi, int steps, uint64_t seed,
                                fmm_cost_model_info *info);
/* The measured autotuner for N_crit (Results section: N_crit is set so that the
 * near- and far-field loads balance; the hybrid selection reduces but does not
 * remove the dependence, because the expansion passes scale with the number of
 * cells).  Solves the given system once per candidate with the options' M2L
 * precision and selection mode, times each solve with events (best of two after
 * a sizing solve) and returns the fastest candidate in *best; ms[k] (may be
 * NULL) receives candidate k's time.  Outputs of the solves are discarded. */
fmm_status fmm_tune_ncrit(const float *xyz, const float *q, int64_t N, int p, double theta, void *stream,
                          const fmm_options *opt, const int *candidates, int ncand, float *ms, int *best);
/* The measured autotuner for the schedule of a solve, single or batched
 * (offsets = NULL for one system of N particles, else the host offsets of
 * fmm_laplace3d_batched with N = offsets[nsys]): every pair of an N_crit
 * candidate and an M2L work-unit size candidate (0 = automatic) is solved and
 * timed with events (best of two after a sizing solve); ms[k * nunit + u] (may
 * be NULL) receives the time of pair (k, u), *best_ncrit and *best_unit the
 * fastest pair.  Outputs of the solves are discarded. */
fmm_status fmm_tune_schedule(const float *xyz, const float *q, int64_t N, const int64_t *offsets, int nsys,
                             int p, double theta, void *stream, const fmm_options *opt, const int *ncrit_cand,
                             int nncrit, const int *unit_cand, int nunit, float *ms, int *best_ncrit,
                             int *best_unit);
/* Parameters as FP32 values: master != 0 gives the FP32 master copy, else the
 * FP16 copy the forward pass uses.  params holds n >= FMM_COST_MODEL_PARAMS floats. */
fmm_status fmm_cost_model_get(float *params, int64_t n, int master);
/* Sets the parameters (n == FMM_COST_MODEL_PARAMS, finite): master copy = params,
 * forward copy = params rounded to FP16; the Adam state is reset. */
fmm_status fmm_cost_model_set(const float *params, int64_t n);
/* Loss and gradient (w.r.t. the FP16 parameters) over a host batch x[B][4],
 * t[B][2], m[B][2], computed by the GPU kernels; no update. */
fmm_status fmm_cost_model_grad(const float *x, const float *t, const float *m, int64_t B, float *loss,
                               float *grad);
/* One Adam step on a host batch; *loss = the loss before the step. */
fmm_status fmm_cost_model_adam_step(const float *x, const float *t, const float *m, int64_t B, float lr,
                                    float *loss);
/* Predictions y[B][2] for host features x[B][4]. */
fmm_status fmm_cost_model_predict(const float *x, int64_t B, float *y);
/* The samples of the last fmm_cost_model_train: *n receives their number; with
 * non-NULL buffers of capacity >= n samples, x[n][4], t[n][2], m[n][2] are copied. */
fmm_status fmm_cost_model_samples(float *x, float *t, float *m, int64_t capacity, int64_t *n);

/* Morton keys and sorted order of the particles, allocating nothing.
 * (The paper has no counterpart: it is a library convenience.)  For callers
 * that must not allocate device memory after start-up -- code running under
 * another framework's memory pool, or a plugin host that forbids cudaMalloc
 * once initialised -- this runs the first stage of fmm_laplace3d (bounding box,
 * FP64 quantisation, 63-bit Morton keys, stable radix sort by key then index)
 * with all scratch in one fixed device array compiled into the library.
 *   xyz   device float32 [N][3], N in [1, 1048576] (larger N: FMM_ERR_ARG)
 *   keys  device uint64 [N]  out: keys in ascending (key, index) order
 *   order device int32 [N]   out: original index of each sorted position
 *   box   device double [4]  out: lo_x, lo_y, lo_z, side of the cubic box
 * Results equal FMM_EXPORT_KEYS / FMM_EXPORT_ORDER / FMM_EXPORT_BOX of a
 * solve on the same points.  A NaN/Inf coordinate gives FMM_ERR_NONFINITE.
 * The scratch array is 16,786,176 bytes.  It is placed in a device's memory
 * when the library's module is loaded on that device; under CUDA's lazy module
 * loading (the default since CUDA 12.2) that happens at the first use of the
 * module there -- in practice the set-up of this entry point's first call on
 * the device (cudaGetSymbolAddress), together with the code of the kernels it
 * launches -- not when the library is loaded into the process.  So the FIRST
 * call on each device does take device memory: a caller that may not allocate
 * after start-up makes one call per device during its initialisation, before
 * any stream capture begins.  From then on the array stays until the process
 * exits, and later calls allocate nothing.  All calls share the array and it
 * keeps the last call's contents (whatever must start at zero is cleared on
 * every call), so calls whose GPU work overlaps (on different streams or
 * threads) race and must be serialised by the caller.  The call synchronises
 * `stream` before returning. */
fmm_status fmm_morton_sort_noalloc(const float *xyz, int64_t N, uint64_t *keys, int32_t *order,
                                   double *box, void *stream);

/* N_crit from the learned cost model (the paper's section "Results" balances
 * the near and far fields through N_crit; the library's network takes that
 * choice without timing the candidates).  For each candidate the library builds
 * the tree, the interaction lists, the offset classes and the M2L tiles of the
 * system (with the options' selection mode; no operator is built, no expansion
 * is evaluated and the candidate is not timed), bins the P2P pairs by the count
 * buckets of the selection table, and sums the network's predicted time per
 * pair over the bins, the number of (tile, class) M2L blocks times a measured
 * time per block, and the number of cells times a measured time per cell.  The
 * cell term is the part of a solve that grows as N_crit shrinks: tree levels,
 * traversal, upward and downward passes, class and tile building.  Both are
 * measured once per (p, theta, precision) and device on an artificial Plummer
 * sphere of 2^20 particles solved at N_crit 32 and 128: the M2L kernel's time
 * over its blocks, and the slope of the time outside the P2P and M2L kernels
 * over the cell count.  The network's P2P sum is scaled so that it equals the
 * P2P kernel's measured time on those two solves.
 * pred_ms[k] (may be NULL) receives candidate k's prediction in ms and *best
 * the candidate with the smallest one.  The measured autotuner (fmm_tune_ncrit)
 * remains the fallback and the judge.  Needs a trained or set model (else
 * FMM_ERR_ARG).  Synchronises `stream`. */
fmm_status fmm_cost_model_pick_ncrit(const float *xyz, const float *q, int64_t N, int p, double theta, void *stream,
                                     const fmm_options *opt, const int *candidates, int ncand, float *pred_ms,
                                     int *best);

/* Ceilings of the FP32 pipe on the current device, for the P2P roofline (the
 * paper has no counterpart; its section "Advantage of N-body algorithms on
 * GPUs" states peaks from the data sheet).  Runs, on `stream`, a kernel of
 * independent FP32x2 FMA chains and the P2P kernel's interaction code on
 * sources staged once in shared memory (no list walk), each timed with events
 * after a warm-up; synchronises `stream`.
 *   ffma_tflops       FMA-stream rate in TFLOP/s (FMA = 2 flop)
 *   body_inter_per_s  interactions per second of the P2P body alone
 * Either pointer may be NULL. */
fmm_status fmm_measure_fp32(double *ffma_tflops, double *body_inter_per_s, void *stream);

/* ---------------------------------------------------------------- captured plans
 * A plan is a solve whose every size lives on the device, captured once into a
 * CUDA graph and replayed for new particle data with one graph launch: no host
 * read-back, no synchronisation, one launch for all systems of the plan (the
 * paper has no counterpart; it is the batched, graph-captured form of the
 * solve).  fmm_plan_create runs one ordinary solve of (xyz, q) to learn the
 * sizes, gives every buffer that size times `headroom` (1 <= headroom <= 16,
 * 0 = 1.25) plus a margin, copies the offset-class operators built so far on
 * the device into the plan (those of this solve among them), and captures the
 * graph.  The plan owns its device memory and its particle and result buffers.
 *
 * A replay whose tree, lists, classes, tiles or work units need more than the
 * capacities, or that meets an offset class with no operator in the plan, is
 * invalid: its results are unspecified (every step stays inside its buffers)
 * and fmm_plan_check returns FMM_ERR_CAPACITY; make a new plan for such data.
 *
 *   offsets  HOST int64 [nsys + 1] as for fmm_laplace3d_batched, or NULL for one
 *            system of N particles (then nsys must be 1)
 *   xyz, q   DEVICE inputs of the first solve (copied into the plan)
 *   stream   the first solve runs on it; creation synchronises it
 * Errors: FMM_ERR_ARG as for the solves (and bad headroom), FMM_ERR_NOMEM, and
 * any error of the first solve. */
typedef struct fmm_plan fmm_plan;
fmm_status fmm_plan_create(fmm_plan **plan, const float *xyz, const float *q, int64_t N, const int64_t *offsets,
                           int nsys, int p, double theta, int ncrit, const fmm_options *opt, double headroom,
                           void *stream);
/* One replay on `stream`, fully asynchronous: copies xyz/q (DEVICE, N values
 * of the plan's layout) into the plan unless they are the plan's own buffers,
 * launches the graph, and copies the results to phi/grad unless they are the
 * plan's own buffers.  Any of the four pointers may be NULL (the plan's buffer
 * is used as it is).  Replays of one plan must be ordered (one stream, or
 * events); the plan must be used on the device it was created on. */
fmm_status fmm_plan_execute(fmm_plan *plan, const float *xyz, const float *q, float *phi, float *grad,
                            void *stream);
/* Synchronises `stream` and reports the last replay: FMM_OK, FMM_ERR_CAPACITY
 * (a capacity was exceeded or a class was unknown; the results are invalid),
 * FMM_ERR_NONFINITE, or FMM_ERR_TIMEOUT. */
fmm_status fmm_plan_check(fmm_plan *plan, void *stream);
/* The plan's own device buffers: xyz float[N][3], q float[N] (inputs) and phi
 * float[N], grad float[N][3] (outputs of the last replay).  Any may be NULL. */
fmm_status fmm_plan_buffers(fmm_plan *plan, float **xyz, float **q, float **phi, float **grad);

typedef struct {
    int64_t N;
    int nsys, levels;                     /* tree levels the graph covers (root = 0) */
    int64_t cell_cap, tile_cap, class_cap, entry_cap, unit_cap;
    int64_t m2l_cap, p2p_cap;             /* interaction-list capacities (pairs) */
    int64_t operators;                    /* offset-class operators held by the plan */
    int64_t graph_nodes, graph_kernels;   /* nodes of the captured graph, kernel nodes among them */
    int64_t last_cells, last_leaves, last_classes, last_entries, last_units;  /* sizes of the last replay */
    int last_valid;                       /* 1 if no capacity was exceeded in the last replay */
} fmm_plan_info_t;
/* Capacities of the plan and the sizes of its last replay (synchronises with
 * the device). */
fmm_status fmm_plan_info(fmm_plan *plan, fmm_plan_info_t *info);
void fmm_plan_destroy(fmm_plan *plan);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char *fmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_FMM_H */
