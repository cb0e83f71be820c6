/*
 * hwfv1.h -- C ABI of the GB300 library for the adaptive Haar-wavelet
 * first-order finite-volume shallow-water model (HWFV1) of Chowdhury,
 * Kesserwani, Rouge & Richmond, arXiv 2206.05761.
 *
 * One timestep of HWFV1 (Algorithm 3) is, in this order:
 *   hwfv1_encode    Haar encoding of the finest h, hu, hv up the hierarchy
 *                   and threshold flags (Eq. 3a-3d, Algorithm 1)
 *   hwfv1_flag      regularised significance tree
 *   hwfv1_traverse  leaf cells of the tree, compacted in Z-order
 *                   (Algorithm 5, Sec. 2.2.3)
 *   hwfv1_step      FV1 update of every leaf from its same-level neighbours
 *                   (Eq. 1-2, Sec. 2.1.3, Sec. 2.2.3)
 *   hwfv1_decode    leaf values back onto the finest grid (Eq. 4 with zero
 *                   details below the leaves) and time advance with the new
 *                   CFL timestep (end of Algorithm 3's time loop)
 * hwfv1_advance runs that sequence for many steps.
 *
 * Conventions
 *  - Every call is asynchronous on the CUDA stream given to hwfv1_init
 *    unless it says it synchronises.  Pointers documented as "device" must
 *    be device memory of the current CUDA device; "host" pointers are read
 *    or written before the call returns.
 *  - Fields exchanged with the caller are float64, row-major over the
 *    finest 2^L x 2^L grid: element (i, j) at j*2^L + i, i along x, j along
 *    y.  The caller owns every pointer it passes; the handle owns all its
 *    internal buffers and frees them in hwfv1_destroy.
 *  - Errors are returned as hwfv1_status.  A bad problem description fails
 *    in hwfv1_init before any device memory is touched.  Conditions found
 *    on the device (non-finite values) are latched and returned by the next
 *    call that synchronises (hwfv1_get_time, hwfv1_advance with
 *    synchronisation, hwfv1_save); hwfv1_last_error gives a message.
 *  - hwfv1_init allocates the handle's buffers; the step, its phases, the
 *    getters (hwfv1_get_fields into host memory aside: a staging area,
 *    returned before it ends), hwfv1_save and hwfv1_load allocate nothing.  A mode's first
 *    use allocates the buffers it adds, once per handle: uniform FV1
 *    (hwfv1_advance_uniform), the learned skip (hwfv1_set_skipnet,
 *    hwfv1_set_skip_levels) and the exact leaf-value store
 *    (hwfv1_set_leaf_store).  hwfv1_batch_init and
 *    the network calls (hwfv1_skipnet_*) allocate their own.  No call
 *    falls back to a CPU computation.
 */
#ifndef HWFV1_H
#define HWFV1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HWFV1_OK = 0,
    HWFV1_ERR_INVALID_SPEC = 1, /* problem description or argument rejected */
    HWFV1_ERR_OOM = 2,          /* device allocation failed                 */
    HWFV1_ERR_CUDA = 3,         /* a CUDA call failed                       */
    HWFV1_ERR_NONFINITE = 4,    /* a non-finite value appeared on the device */
    HWFV1_ERR_NEG_DEPTH = 5,    /* reserved: negative depth in an input     */
    HWFV1_ERR_TIMEOUT = 6,      /* reserved: a bounded device wait ran out  */
    HWFV1_ERR_STATE = 7         /* call not valid in the handle's state      */
} hwfv1_status;

/* Boundary kinds (Sec. 3 test cases use closed walls, open boundaries and
 * an inflow boundary). */
typedef enum {
    HWFV1_BC_CLOSED = 0,        /* reflective wall: ghost = cell, normal q negated */
    HWFV1_BC_TRANSMISSIVE = 1,  /* open boundary: ghost = copy of the cell         */
    HWFV1_BC_INFLOW = 2         /* wall plus a volume source Q(t) on the inlet     */
} hwfv1_bc_kind;

/* Regularisation switches (hwfv1_problem.flags). */
#define HWFV1_REG_PREDICT 1u    /* children of a significant detail become significant */
#define HWFV1_REG_CLOSE 2u      /* ancestors of a significant detail become significant */
/* Execution switch (no counterpart in the paper; results are identical with
 * and without it): update every leaf each step.  Without it, a step skips
 * the tiles of 32 x 32 finest cells whose state is +0 in both state buffers
 * and next to tiles at +0 (dry ground far from water): their update would
 * reproduce the values already stored.  Skipping is off when eps < 1e-30
 * (thresholds that round to 0 flag zero details). */
#define HWFV1_FULL_SWEEP 4u
/* Conservative variant (a switch of this library; the paper's update uses
 * the same-level neighbour on every face, Sec. 2.1.3, which does not
 * conserve mass where the resolution changes).  A face of a leaf whose
 * same-level neighbour is refined (smaller leaves lie behind it) takes, for
 * its flux and for the leaf's own reconstructed depth squared in the bed
 * source term, the average of its two halves one level finer, recursively,
 * down to the half faces whose neighbour cell is a leaf; each such half face
 * is evaluated between the two same-level cells that touch it, as the
 * smaller leaf evaluates it.  Both sides of every face then carry one flux:
 * mass is conserved up to rounding on closed domains whose finest depths
 * hand a leaf's volume down unchanged.  Needs HWFV1_REG_CLOSE; single
 * domains only (not hwfv1_batch_init, not with hwfv1_set_skipnet). */
#define HWFV1_FLUX_MATCH 8u

/* Problem description.  The user inputs of Algorithm 3 are L and eps (t_end
 * is given to hwfv1_advance); CFL = 0.5 is the paper's choice (Sec. 2.1.3).
 * All lengths in metres, times in seconds. */
typedef struct hwfv1_problem {
    double x0, y0;       /* domain origin                                         */
    double lx, ly;       /* domain extent (> 0); finest cell dx = lx/2^L           */
    double eps;          /* error threshold: 0, or in [1e-200, 1e300]             */
    double cfl;          /* Courant number in (0, 1]                              */
    double g;            /* gravitational acceleration (> 0)                      */
    double manning_n;    /* Manning coefficient (>= 0; 0 = frictionless), Eq. 1   */
    double tol_h;        /* wet/dry depth tolerance (> 0)                         */
    double dt_max;       /* largest timestep, also the step when all is dry (> 0) */
    int32_t L;           /* maximum refinement level, 1..14                       */
    int32_t precision;   /* 64 (parity path) or 32                                */
    int32_t bc[4];       /* hwfv1_bc_kind of the W, E, S, N sides                 */
    int32_t inflow_a0;   /* inflow side: finest cells [a0, a1) along the side     */
    int32_t inflow_a1;   /*   (j for W/E, i for S/N)                              */
    int32_t inflow_n;    /* number of hydrograph points (>= 1 with an inflow side) */
    uint32_t flags;      /* HWFV1_REG_* bits                                       */
    const double* inflow_t; /* host, inflow_n strictly increasing times           */
    const double* inflow_Q; /* host, inflow_n discharges (m^3/s); Q(t) is
                               piecewise linear, constant outside the range      */
} hwfv1_problem;

typedef struct hwfv1_handle hwfv1_handle;

/* Create a simulation from the initial finest fields (row-major, float64,
 * 4^L elements each; qx = hu, qy = hv) and bed z.  Each of the four may be
 * device memory or host memory (pinned or pageable): a host field is copied
 * to the device on a stream of the handle's own, in the order z, h, qx, qy,
 * through a staging area of 2 x 4^L doubles taken from the device pool and
 * returned before the call ends, so that the bed is converted and encoded
 * while the other fields are still being copied.  Copies the fields into
 * the handle's Morton-ordered hierarchy, encodes the static bed once, sets
 * t = 0 and dt from the CFL condition on the initial state, and captures
 * the plain step's graphs (which hwfv1_advance launches).  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Synchronises: the caller's
 * buffers are no longer read when it returns.
 * Initial discretisation: the first step of Algorithm 3. */
hwfv1_status hwfv1_init(const hwfv1_problem* spec, const double* z, const double* h,
                        const double* qx, const double* qy, void* stream,
                        hwfv1_handle** out);

/* The phases of one plain step, one call each (encode, flag, traverse,
 * step, decode); hwfv1_advance runs them in one graph.  While the learned
 * subtree skip is on they return HWFV1_ERR_STATE (the stored state may be
 * above level L there).
 * Encoding (Eq. 3a-3d, Algorithm 1): scaling coefficients of h, hu, hv for
 * every level below L from the finest grid, threshold flags of every
 * parent against the normalised threshold 2^(n-L)*eps*s_max (Sec. 2.1.2),
 * and the upward closure of those flags. */
hwfv1_status hwfv1_encode(hwfv1_handle* hd);

/* Regularised significance: the encoded flags joined with the bed's
 * (static) flags, the children of every significant detail, and (with
 * HWFV1_REG_CLOSE) every ancestor of a significant detail. */
hwfv1_status hwfv1_flag(hwfv1_handle* hd);

/* Leaf cells of the significance tree (Algorithm 5: a finest cell's walk
 * from the root stops at the first insignificant detail or at level L),
 * duplicates removed by stream compaction (Sec. 2.2.3), in Z-order.  If
 * num_leaves is not NULL the count is written there (host) and the call
 * synchronises; otherwise it stays on the device. */
hwfv1_status hwfv1_traverse(hwfv1_handle* hd, int64_t* num_leaves);

/* FV1 forward-Euler update (Eq. 2) of every leaf with L_c built from the
 * leaf's coefficients and its same-level neighbours' (Sec. 2.1.3): HLL
 * fluxes with hydrostatic reconstruction, bed slope, Manning friction,
 * inflow source; reduces the CFL bound of the updated leaves. */
hwfv1_status hwfv1_step(hwfv1_handle* hd);

/* Decode-back: every finest cell under a coarser leaf takes the leaf's
 * discharges and free surface (Eq. 4 with zero details below leaves);
 * then t += dt and the next dt = CFL * (min CFL bound) (end of
 * Algorithm 3's time loop), clamped so that no step passes the t_end of hwfv1_advance. */
hwfv1_status hwfv1_decode(hwfv1_handle* hd);

/* Run up to max_steps full steps (encode, flag, traverse, step, decode),
 * stopping at t_end: a step never passes t_end and steps after it are
 * no-ops.  Captures one step in a CUDA graph on first use and replays it.
 * Does not synchronise. */
hwfv1_status hwfv1_advance(hwfv1_handle* hd, double t_end, int64_t max_steps);

/* The same time loop with uniform FV1 on the finest grid: every finest cell
 * is updated from its four finest neighbours every step, with no encode,
 * flag, traversal or decode (eps plays no part).  This is the GPU-FV1
 * solver the paper compares HWFV1 against (Sec. 3); it reproduces HWFV1
 * with eps = 0.  The state stays the finest fields, so the two loops can be
 * mixed on one handle.  Allocates a list of the 4^L finest cells on first
 * use.  Does not synchronise. */
hwfv1_status hwfv1_advance_uniform(hwfv1_handle* hd, double t_end, int64_t max_steps);

/* Current finest fields h, hu, hv (row-major float64, 4^L each; any pointer
 * may be NULL).  An output may be device or host memory (pinned or
 * pageable).  Host outputs are formed in a staging area of 2 x 4^L doubles
 * from the device pool (returned before the call ends) and copied out one
 * field while the next is formed; the call then synchronises, and the host
 * outputs are written when it returns.  With device outputs only it is
 * asynchronous and allocates nothing. */
hwfv1_status hwfv1_get_fields(hwfv1_handle* hd, double* h, double* qx, double* qy);

/* Replace the finest h, hu, hv (device, row-major float64) keeping t and dt;
 * s_max is recomputed from the new fields. */
hwfv1_status hwfv1_set_fields(hwfv1_handle* hd, const double* h, const double* qx,
                              const double* qy);

/* Leaves of the last traversal (device output, `cap` uint32 entries), each
 * packed as (level << 28) | Morton code within the level, in Z-order of
 * their first finest cell.  *n (host) receives the count.  Synchronises.
 * Returns HWFV1_ERR_INVALID_SPEC if cap is too small (nothing written). */
hwfv1_status hwfv1_get_leaves(hwfv1_handle* hd, uint32_t* packed, int64_t cap, int64_t* n);

/* Significance bits (device output).  which = 0: threshold flags of
 * h, hu, hv and z (Algorithm 1's threshold test); 1: regularised flags used by the
 * traversal.  Level n (0..L-1) occupies words [w(n), w(n+1)) with w(n) = n
 * for n <= 3 and 3 + (4^n - 64)/96 above; bit b of word k of level n is
 * the parent with Morton code 32k + b.  `cap_words` must be >= w(L). */
hwfv1_status hwfv1_get_flags(hwfv1_handle* hd, int32_t which, uint32_t* bits, int64_t cap_words);

/* Encoded coefficients of one level (device output, float64, 4^level
 * values in Morton order).  field: 0 h, 1 hu, 2 hv, 3 z. */
hwfv1_status hwfv1_get_level(hwfv1_handle* hd, int32_t field, int32_t level, double* out);

/* Time, next timestep and number of steps taken (host outputs, any may be
 * NULL).  Synchronises and reports latched device errors. */
hwfv1_status hwfv1_get_time(hwfv1_handle* hd, double* t, double* dt, int64_t* step);

/* Set the time and the timestep of the next step (dt > 0). */
hwfv1_status hwfv1_set_time(hwfv1_handle* hd, double t, double dt);

/* Diagnostics of the last completed step (host outputs, synchronises):
 * number of leaves and the maxima of |h|, |hu|, |hv| used for s_max. */
hwfv1_status hwfv1_get_stats(hwfv1_handle* hd, int64_t* num_leaves, double* smax3);

/* One step (encode .. time advance: the step hwfv1_advance takes next, the
 * plain step outside the learned skip) with a CUDA event recorded after
 * every kernel: the step is captured as a graph
 * whose kernels are separated by event-record nodes (HWFV1_NO_GRAPH set:
 * ordinary launches on the handle's stream).  Writes the duration in ms of
 * each kernel (from the previous event) to ms[0..cap) and its name (static
 * strings owned by the library) to names[0..cap); either may be NULL;
 * *n = number of kernels.  Advances the simulation by one step and
 * synchronises.  No counterpart in the paper: diagnostics. */
hwfv1_status hwfv1_profile_step(hwfv1_handle* hd, float* ms, const char** names, int32_t cap, int32_t* n);

/* One plain step whose full update of the queued (wet) leaves, Eq. 2 on the
 * leaf grid, is captured on its own and replayed `reps` (>= 1) times between
 * two CUDA events on the handle's stream before the step goes on
 * (HWFV1_ERR_STATE while the learned skip is on).  Every
 * replay reads the same state and queue and writes the same values (leaf
 * values of the next state, min/max reductions), so the simulation still
 * advances by exactly one step.  *ms (host) = the mean time of one update,
 * the kernels as they run inside the step's graph.  Synchronises.  No
 * counterpart in the paper: diagnostics. */
hwfv1_status hwfv1_profile_update(hwfv1_handle* hd, int32_t reps, float* ms);

/* Measured FP64 add throughput of the current device (host output, TFLOP/s
 * at one FLOP per instruction): a grid of 8 CTAs of 256 threads per SM,
 * each thread running eight independent chains of dependent double
 * additions, timed with CUDA events, best of three after a warm-up.  The
 * wet-leaf update is bound by this pipe.  No counterpart in the paper:
 * diagnostics.  Synchronises; allocates and frees a small buffer. */
hwfv1_status hwfv1_fp64_throughput(double* tflops);

/* Running counters (host outputs, any may be NULL; synchronises): steps
 * taken; leaves updated summed over those steps (sum of M, the work of
 * Sec. 2.3's leaf loop); the part of them outside skipped quiescent tiles
 * (see HWFV1_FULL_SWEEP), i.e. the leaves the kernels touched; the part
 * that took the full FV1 update (not entirely dry); and the number of
 * kernels one captured step launches (the learned step's when a network is
 * attached; capturing the graph here if no step has run yet).  No
 * counterpart in the paper: diagnostics. */
hwfv1_status hwfv1_get_counters(hwfv1_handle* hd, int64_t* steps, int64_t* leaf_updates,
                                int64_t* active_updates, int64_t* wet_updates, int64_t* kernels_per_step);

/* Checkpoint: the finest h, hu, hv (Morton order, the handle's precision),
 * t, dt and the step count, written to a host buffer.  With host_buf NULL
 * only *used is set to the size needed.  Synchronises. */
hwfv1_status hwfv1_save(hwfv1_handle* hd, void* host_buf, size_t cap, size_t* used);

/* Restore a checkpoint written by hwfv1_save for the same problem. */
hwfv1_status hwfv1_load(hwfv1_handle* hd, const void* host_buf, size_t n);

/* Message of the last error on this handle ("" if none). */
const char* hwfv1_last_error(hwfv1_handle* hd);

/* Free all device memory of the handle.  The handle's buffers come from
 * the device's default stream-ordered memory pool (cudaMallocAsync on the
 * handle's stream), whose release threshold the library sets to keep freed
 * memory for the next handle; cudaMemPoolTrimTo on that pool returns it to
 * the device. */
void hwfv1_destroy(hwfv1_handle* hd);

/* ------------------------------------------------------------------------
 * Learned subtree skip (a layer this library adds; the paper has no learned
 * part).  The paper's significance tree (Sec. 2.1.2, Fig. 2) is built from
 * every detail down to the finest level each step.  Here each level-(L-4)
 * cell's subtree (16 x 16 finest cells) is given a predicted level p, the
 * deepest level it needs: the subtree is encoded only from its storage
 * level, its details below p are neither formed nor tested, its leaves are
 * no finer than p, and its state is stored at P = the largest p of itself
 * and its four edge neighbours (so a neighbouring leaf finds its
 * same-level cell there); a coarser stored subtree moves 4^(P-L) of the
 * bytes of the finest one.  Every audit_K-th step is the exact (plain)
 * step of the whole finest grid.  The levels come from a small CNN
 * (3 layers of 3x3 convolutions, 4 -> 16 -> 16 -> 5 channels, ReLU, BF16
 * weights and activations, FP32 accumulation on the tensor cores) that
 * reads the level-(L-4) coefficients of h, hu, hv, z (each over its s_max)
 * of the state a step has just encoded and predicts, per subtree, the
 * deepest level the next step's threshold tree will need; or from the
 * caller (hwfv1_set_skip_levels).
 * Parameters are FP32 in the layout w1[16][4][3][3], b1[16], w2[16][16][3][3],
 * b2[16], w3[5][16][3][3], b3[5] (hwfv1_skipnet_num_params() floats).
 * ------------------------------------------------------------------------ */
typedef struct hwfv1_skipnet hwfv1_skipnet;

int32_t hwfv1_skipnet_num_params(void);
/* New network with seeded He-initialised weights (device memory). */
hwfv1_status hwfv1_skipnet_create(uint32_t seed, hwfv1_skipnet** out);
hwfv1_status hwfv1_skipnet_set_params(hwfv1_skipnet* net, const float* host, int64_t n);
hwfv1_status hwfv1_skipnet_get_params(hwfv1_skipnet* net, float* host, int64_t n);
/* Logits of nimg images x (device, bf16 bits, [nimg][H][W][4] channels
 * last) into logits (device, float, [nimg*H*W][16], classes 0..4 valid).
 * Synchronises; HWFV1_ERR_TIMEOUT if a tensor-core wait ran out. */
hwfv1_status hwfv1_skipnet_forward(hwfv1_skipnet* net, const uint16_t* x, int32_t nimg, int32_t H, int32_t W,
                                   float* logits);
/* Mean softmax cross-entropy (host *loss) and its gradient (host grads,
 * hwfv1_skipnet_num_params() floats) for labels (device, uint8 per pixel,
 * classes 0..4).  Synchronises. */
hwfv1_status hwfv1_skipnet_gradients(hwfv1_skipnet* net, const uint16_t* x, const uint8_t* labels, int32_t nimg,
                                     int32_t H, int32_t W, double* loss, float* grads);
/* Adam training over nimg images in minibatches of `batch` images (shuffled
 * by batch with `seed`) for `epochs`; *last_loss (host) gets the loss of the
 * last minibatch.  Synchronises. */
hwfv1_status hwfv1_skipnet_train(hwfv1_skipnet* net, const uint16_t* x, const uint8_t* labels, int32_t nimg,
                                 int32_t H, int32_t W, int32_t batch, int32_t epochs, float lr, uint32_t seed,
                                 double* last_loss);
void hwfv1_skipnet_destroy(hwfv1_skipnet* net);

/* Use `net` (NULL: stop) for the learned subtree skip of hwfv1_advance.
 * Counting from the next step, every audit_K-th step (>= 1) is the exact
 * plain step and the others are skip steps.  A subtree's predicted level is
 * L-4 plus the smallest class whose predicted cumulative probability
 * reaches 1 - margin (margin < 0 keeps level L everywhere, which is the
 * plain method).  The network runs on the audit step and on every
 * predict_every-th (>= 1) step after it within an audit interval, after the
 * step's encode, and its levels serve the steps that follow; the steps in
 * between reuse them.  Needs L >= 6, HWFV1_REG_PREDICT and HWFV1_REG_CLOSE,
 * not HWFV1_FLUX_MATCH.  Stopping brings the stored state to level L.  The
 * network must outlive its use. */
hwfv1_status hwfv1_set_skipnet(hwfv1_handle* hd, hwfv1_skipnet* net, int32_t audit_K, float margin,
                               int32_t predict_every);
/* The learned subtree skip with levels given by the caller instead of the
 * network: `levels` (host, 4^(L-4) bytes, row-major over level L-4, j
 * major, each in [L-4, L]; NULL: stop) is kept for every skip step until
 * the next call; audit_K as above.  Needs L >= 5 (and the flags above).
 * HWFV1_ERR_INVALID_SPEC for a level out of range. */
hwfv1_status hwfv1_set_skip_levels(hwfv1_handle* hd, const uint8_t* levels, int32_t audit_K);
/* Exact leaf-value store (on = 1; 0 stops it).  The paper's encoding runs
 * only along the tree of significant details (the note after Algorithm 3);
 * here, exactly: a level-(L-4) subtree whose bed is flat (every finest bed
 * value equal) is stored at its deepest leaf level m instead of the finest
 * grid.  Every finest cell below a stored cell then holds that cell's value
 * (the decode-back hands a leaf's value, with its free surface, to every
 * finest cell below it), so the subtree's details at levels >= m are zero and
 * flag nothing (eps > 0): it is encoded from level m only, kept down to
 * m + 1 (where its next leaves can be), and its coarse leaves are decoded
 * down to level m, not L.  Other subtrees are stored at L.  Results are the
 * plain step's bit for bit; the bytes a flat subtree moves fall as
 * 4^(m-L).  Quiescent-tile skipping (HWFV1_FULL_SWEEP) does not apply while
 * it is on.  Needs L >= 5, eps >= 1e-30, HWFV1_REG_PREDICT and
 * HWFV1_REG_CLOSE, not HWFV1_FLUX_MATCH; not together with the learned
 * skip (turning one on turns the other off).  hwfv1_get_skip_levels(1)
 * gives the storage levels. */
hwfv1_status hwfv1_set_leaf_store(hwfv1_handle* hd, int32_t on);
/* which = 0: the predicted levels in use; which = 1: the level each
 * subtree's state is stored at (L outside the skip).  Host output, 4^(L-4)
 * bytes, row-major over level L-4.  Synchronises. */
hwfv1_status hwfv1_get_skip_levels(hwfv1_handle* hd, int32_t which, uint8_t* out, int64_t cap);
/* CNN input of the current state (device output, bf16 bits, 4 x 4^(L-4)
 * values, channels last, row j of subtrees major); call after hwfv1_encode. */
hwfv1_status hwfv1_get_features(hwfv1_handle* hd, uint16_t* out, int64_t cap);
/* Training label of every subtree for the current state (device output,
 * uint8 per subtree, row-major): 1 + the deepest level >= L-4 holding a
 * closed threshold flag, minus (L-4); 0 if none.  Call after hwfv1_encode. */
hwfv1_status hwfv1_get_labels(hwfv1_handle* hd, uint8_t* out, int64_t cap);

/* ------------------------------------------------------------------------
 * Batched ensembles: many independent domains (each its own problem, its
 * own L, its own t and dt) advanced together.  Every phase of a step is one
 * launch over all domains (a flat grid mapped onto (domain, block) through a
 * per-domain block table) and one ensemble step is one CUDA graph.  The
 * paper runs one domain; this is the batched form of the same path.
 * ------------------------------------------------------------------------ */
typedef struct hwfv1_batch hwfv1_batch;

/* n problems (all with the same precision) and their initial fields (arrays
 * of n device pointers, each field as in hwfv1_init).  Synchronises. */
hwfv1_status hwfv1_batch_init(const hwfv1_problem* specs, int32_t n, const double* const* z,
                              const double* const* h, const double* const* qx,
                              const double* const* qy, void* stream, hwfv1_batch** out);

/* Up to max_steps ensemble steps; each domain stops at t_end (its later
 * steps are no-ops).  Does not synchronise. */
hwfv1_status hwfv1_batch_advance(hwfv1_batch* b, double t_end, int64_t max_steps);

/* Time trial_steps ensemble steps under each candidate launch configuration
 * (encode levels per pass in {5,4,3}, finest cells per FV1 thread in
 * {8,32,128,512}; with 5, the first pass of a member of L >= 8 covers
 * 1024-cell blocks but stops three levels up) and keep the fastest; choice
 * (host, 2 int32, may be NULL)
 * receives it.  All candidates give bit-identical results; the trials
 * advance the ensemble by 12 x (trial_steps + 1) steps.  Synchronises. */
hwfv1_status hwfv1_batch_autotune(hwfv1_batch* b, int64_t trial_steps, int32_t* choice);

/* Handle of member d for the single-domain getters (hwfv1_get_fields,
 * hwfv1_get_time, hwfv1_get_leaves, ...).  The batch owns it: hwfv1_destroy
 * on it does nothing; it is freed by hwfv1_batch_destroy. */
hwfv1_status hwfv1_batch_member(hwfv1_batch* b, int32_t d, hwfv1_handle** view);

/* Kernel launches in one ensemble step (the captured graph's nodes). */
int64_t hwfv1_batch_launches_per_step(hwfv1_batch* b);

const char* hwfv1_batch_last_error(hwfv1_batch* b);
void hwfv1_batch_destroy(hwfv1_batch* b);

/* Leaf list from a regularised significance bit array, for callers that
 * cannot allocate device memory (a host framework whose pool allocator owns
 * the device memory budget, a fixed-footprint deployment, a latency-bound
 * loop that cannot take cudaMalloc's implicit synchronisation).  The paper
 * has no counterpart: it is the traversal and compaction of hwfv1_traverse
 * with its per-tile scratch held in a fixed 128 KiB __device__ array inside
 * the library instead of handle-owned buffers.
 *   sig_bits    device, levels 0..L-1 in the layout of hwfv1_get_flags
 *               (which = 1), at least w(L) words; read only
 *   L           1..12 (the scratch is sized for L <= 12; larger L returns
 *               HWFV1_ERR_INVALID_SPEC)
 *   leaves      device output, `cap` entries, packed as in hwfv1_get_leaves;
 *               leaves past cap are not written
 *   num_leaves  device output, one uint32: the number of leaves (may exceed
 *               cap, so the caller can tell the list was cut)
 *   stream      cudaStream_t the three kernels run on (asynchronous)
 * No call allocates memory.  Outside a stream capture every call looks up
 * the scratch array's device address in the current context
 * (cudaGetSymbolAddress, a host-side query that allocates nothing), so a
 * context that was reset or replaced between calls gets the right address;
 * while `stream` is capturing, the address of the last uncaptured call on
 * that device is used, so make the first call on each device before any
 * stream capture.  If an error from an earlier, unrelated call is pending
 * (cudaPeekAtLastError), the call launches nothing, leaves that error
 * pending and returns HWFV1_ERR_CUDA.  All calls share the scratch, so calls
 * that overlap on the GPU (different streams or devices' contexts running
 * concurrently on one device) race; serialise them.  Every scratch word a
 * call reads is written by that call first, so no clearing is needed
 * between calls. */
hwfv1_status hwfv1_traverse_noalloc(const uint32_t* sig_bits, int32_t L, uint32_t* leaves,
                                    int64_t cap, uint32_t* num_leaves, void* stream);

/* Library version, for the loader's sanity check. */
int32_t hwfv1_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HWFV1_H */
