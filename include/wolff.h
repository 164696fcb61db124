/*
 * wolff.h -- C ABI of the GB300 Wolff single-cluster library.
 *
 * The operation (Komura & Okabe, "GPU-based single-cluster algorithm for the
 * simulation of the Ising model", section 2 and section 4):
 *   H = -J sum_<ij> S_i S_j on the periodic L^D lattice, D = 2 (square) or
 *   D = 3 (simple cubic), site i = x + L*y (+ L*L*z).  One single-cluster
 *   update t: pick a random seed site (step (i)); grow the cluster by parallel
 *   expansion of the newly added ("wave-front") spins, each testing its
 *   parallel neighbours with bond probability p = 1 - exp(-2J/T)
 *   (steps (ii)-(iv) and (iii')); flip the finished cluster.
 *
 * Randomness is counter based (Philox4x32-10, Salmon et al. SC'11) with
 * key = (seed mod 2^32, seed >> 32):
 *   bond (o,d) of update t  -> lane d of Philox(ctr = (o, t_lo, t_hi, 0)),
 *   seed site of update t   -> floor(lane0(Philox((0, t_lo, t_hi, 1))) * N / 2^32),
 *   initial spin of site i  -> -1 if bit 31 of lane0(Philox((i, 0, 0, 2))) else +1.
 * A bond is active when its random word is below thr = floor(p * 2^32), p
 * evaluated on the host in IEEE double (the device never evaluates exp).  The
 * cluster is therefore the connected component of the seed in the graph of
 * active bonds joining spins parallel to the seed, whatever order the GPU
 * explores it in, and every result is reproducible bit for bit.
 *
 * Observables: E_bond = sum_{i,d} s_i s_{nb(i,d)} over the D*N forward bonds
 * (physical energy = -J * E_bond) and M = sum_i s_i, both exact integers.
 *
 * Conventions for every entry point:
 *   - Returns a wolff_status; nothing is thrown across the ABI.
 *   - Pointers named d_* are device pointers on the context's device, h_* are
 *     host pointers.  The caller owns every buffer it passes and must keep it
 *     alive until the work using it has completed on the context's stream.
 *   - Device work is enqueued on the stream given to ising_init (NULL = the
 *     legacy default stream) and is asynchronous unless stated otherwise.
 *     Errors detected on the device (a bounded wait that ran out, an invalid
 *     state word) are latched in the context and reported by the next call
 *     that synchronises (measure, measure_full, wolff_get_state, ...).
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef WOLFF_H
#define WOLFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WOLFF_OK = 0,
    WOLFF_EINVAL = 1,         /* bad argument (size, pointer, parameter) */
    WOLFF_ENOMEM = 2,         /* workspace too small or allocation failed */
    WOLFF_ECUDA = 3,          /* a CUDA runtime call failed */
    WOLFF_ETIMEOUT = 4,       /* a device-side bounded wait gave up */
    WOLFF_EUNSUPPORTED = 5    /* valid request this build cannot serve */
} wolff_status;

/* Spin layouts.  INT8: one byte per site (bit 0 = current spin, bit 1 = spin
 * at the start of the running update; +1 is stored as 1). */
enum { WOLFF_LAYOUT_INT8 = 0 };

/* How one update's levels are synchronised (section 3 of the paper replaced):
 *   PERSISTENT  one cooperative launch per wolff_step; all updates and levels
 *               run inside it; CTA 0 grows small wave fronts alone and hands
 *               large ones to every CTA, levels then separated by a bounded
 *               grid-wide barrier;
 *   GRAPH       a CUDA graph: one kernel node per level inside a conditional
 *               WHILE node, nested inside a WHILE node over updates;
 *   CLUSTER     one thread-block cluster (1..16 CTAs) per lattice: CTA 0
 *               grows small fronts alone, larger ones are shared by the
 *               cluster with the hardware cluster barrier between levels;
 *   TINY        Ising lattices of at most WOLFF_TINY_MAX_SITES sites: one CTA
 *               holds the whole lattice in shared memory for the launch, as
 *               bit planes (each row of L sites in ceil(L/32) 32-bit words);
 *               a breadth-first level computes the next wave front of every
 *               word with shifts and masks, and E_bond, M are recounted with
 *               population counts after each flip.  Lattices of at most 64
 *               words (2D L <= 32, 3D L <= 8) with 64 threads or more: warp 0
 *               runs the update alone (__syncwarp per level) while the
 *               other warps draw the next update's bond randomness; larger
 *               ones: every thread grows one or two words (__syncthreads per
 *               level).  The paper's CPU/GPU hybrid (section 5) starts small
 *               clusters on the CPU; here a small lattice never leaves one
 *               SM.  grid_blocks must be 0 or 1; block_threads from 32 to
 *               768 in 2D and 512 in 3D, at least half the lattice's words
 *               unless warp 0 runs alone (EINVAL otherwise);
 *               On lattices above 64 words TINY draws every site's bonds
 *               each update: measured 3-11x faster than CLUSTER while the
 *               clusters are large (equilibrated at or below T_c), up to 72x
 *               slower on clusters of a few sites (random starts, above T_c),
 *               where CLUSTER's window mode grows many updates at once;
 *   AUTO        the library's choice: TINY for Ising lattices of at most 64
 *               words (2D L <= 32, 3D L <= 8; 9-29x faster than CLUSTER in
 *               every regime measured), else CLUSTER with the largest cluster
 *               the GPU launches (16 where non-portable sizes are allowed,
 *               else 8), 512 threads, t_up = 128, t_down = 64, window mode
 *               on.  A new context starts on AUTO's choice; AUTO with
 *               grid_blocks > 1 or a block_threads TINY cannot use means
 *               CLUSTER. */
enum {
    WOLFF_SCHED_AUTO = 0,
    WOLFF_SCHED_PERSISTENT = 1,
    WOLFF_SCHED_GRAPH = 2,
    WOLFF_SCHED_CLUSTER = 3,
    WOLFF_SCHED_TINY = 4
};
#define WOLFF_TINY_MAX_SITES 32768

/* One record per update, written after the update's flip
 * (section 5, the "+ measurement" column of Tables 1-2). */
typedef struct {
    uint32_t C;        /* cluster size |C_t| */
    uint32_t levels;   /* breadth-first generations grown (1 = lone seed) */
    int64_t  E_bond;   /* bond sum after the flip */
    int64_t  M;        /* magnetisation after the flip */
} wolff_record;

/* Static facts about a context. */
typedef struct {
    int      dim, L;
    uint32_t N;            /* L^dim */
    uint64_t thr;          /* bond threshold floor(p 2^32), 0 .. 2^32 */
    uint64_t seed;
    uint64_t t;            /* index of the next update (host mirror) */
    int      schedule;     /* schedule wolff_step will use */
    int      grid_blocks;  /* CTAs of the growth kernels */
    int      block_threads;
    int      sm_count;
    size_t   workspace_bytes;
    int      helper_clusters;  /* pre-growing helper teams a wolff_step of the
                                  cluster schedule launches beside the main one */
} wolff_info;

typedef struct wolff_ctx wolff_ctx;

/* Bytes of device workspace a context of this shape needs (0 if the shape is
 * invalid).  The workspace holds the spin array, the cluster list (the ic/in
 * list of section 2, one 32-bit entry per site) and a small control block;
 * lattices of 2^20 sites or more also get a 4 MiB ring of pre-grown updates
 * (see wolff_set_helpers). */
size_t wolff_workspace_bytes(int dim, int L, int layout);

/* Creates a context on the current device and initialises the lattice from
 * Philox (update counter t = 0), then computes E_bond and M by a full pass.
 * Paper: section 2 (the model H = -J sum S_i S_j on the periodic lattice,
 * and the bond probability p = 1 - exp(-2J/T) of step (ii), whose threshold
 * this computes on the host); the random start is the one of section 5's
 * runs, drawn from Philox instead of the paper's generator.
 *   dim         2 or 3;  L >= 2, with dim*L^dim < 2^32 and L <= 1024 in 3D,
 *               L <= 32767 in 2D;
 *   J, T        coupling and temperature, J >= 0, T > 0 (T may be +inf);
 *   seed        Philox key;  layout  WOLFF_LAYOUT_INT8;
 *   d_workspace device buffer of at least wolff_workspace_bytes(), 256-byte
 *               aligned, owned by the caller, not to be used by anyone else
 *               while the context lives; NULL makes the library cudaMalloc
 *               (and later free) its own;
 *   stream      cudaStream_t to enqueue on (NULL = default stream).
 * On success *out receives the context.  EINVAL for a bad shape/parameter or
 * a misaligned/small workspace, ENOMEM if the library's allocation fails. */
wolff_status ising_init(wolff_ctx **out, int dim, int L, double J, double T,
                        uint64_t seed, int layout, void *d_workspace,
                        size_t workspace_bytes, void *stream);

/* ---- q-state Potts model ------------------------------------------------
 * The extension section 6 of the paper names as straightforward:
 * H = -J sum_<ij> delta(c_i, c_j), colours c in 0..q-1, 2 <= q <= 64.  One
 * update t: seed site from lane 0 of the seed draw and a new colour
 * c' = (c0 + 1 + floor(x1 (q-1) / 2^32)) mod q from lane 1; the cluster grows
 * through bonds to neighbours of colour c0 that are active with
 * p = 1 - exp(-J/T), tested on the same bond words as the Ising update; every
 * member takes c'.  With q = 2 the chain equals the Ising chain of coupling
 * J/2 (colour 1 <-> spin -1).  Initial colour of site i:
 * floor(x q / 2^32), x = lane 0 of Philox(i, 0, 0, 2).
 * A Potts context is used through the same entry points as an Ising one:
 *   - records and measure() report E_bond = the number of satisfied forward
 *     bonds (energy -J E_bond) and, in place of M, N0 = the number of sites
 *     of colour 0;
 *   - wolff_get_state / wolff_set_state exchange colours (int8 0..q-1);
 *     set_state rejects other values with WOLFF_EINVAL;
 *   - only the CLUSTER schedule runs it (no window mode); wolff_batch_run
 *     returns WOLFF_EUNSUPPORTED for Potts contexts.
 * Other arguments and ownership as for ising_init. */
wolff_status potts_init(wolff_ctx **out, int dim, int L, int q, double J, double T,
                        uint64_t seed, void *d_workspace, size_t workspace_bytes,
                        void *stream);

/* ---- XY model (embedded-cluster update) ---------------------------------
 * The model section 6 of the paper names next: H = -J sum_<ij>
 * cos(theta_i - theta_j), updated by Wolff's embedded Ising cluster (Wolff,
 * PRL 62 (1989) 361).  Update t: seed site from lane 0 of the seed draw and
 * a reflection angle phi from lane 1; a bond <ij> is active with probability
 * 1 - exp(-2K (r.s_i)(r.s_j)) when (r.s_i)(r.s_j) > 0 (K = J/T, judged on
 * the pre-update spins, the same bond words as the Ising update); every
 * member of the seed's component is reflected: theta -> pi + 2 phi - theta.
 * Exact integer arithmetic, so that results are reproducible bit for bit:
 *   - angles are integers in units of 2 pi / 65536 on a grid of angle_bits
 *     (1..15) bits: spins are multiples of 2^(16 - angle_bits) and phi of
 *     2^(15 - angle_bits) (15 = the finest; small values give 2^bits-state
 *     clock models);
 *   - cos is the fixed-point table round(cos(pi k / 32768) 2^30), k =
 *     0..16384, extended by symmetry; r.s_i = I(theta_i - phi);
 *   - y = (2K 2^-60) (I_i I_j) in double, p = 1 - e^-y with e^-y from
 *     Cody-Waite range reduction and a degree-16 Taylor series in a fixed
 *     sequence of correctly rounded double operations; the bond is active
 *     when its random word is below floor(p 2^32);
 *   - initial angle of site i: the top angle_bits bits of lane 0 of
 *     Philox(i, 0, 0, 2), shifted to the grid.
 * Records and measurements are fixed point: E = sum_{i,d} I(theta_i -
 * theta_nb(i,d)) (energy -J E 2^-30), Mx = sum I(theta_i), My = sum
 * I(theta_i - 16384).  An XY context runs through wolff_step (d_records
 * receives wolff_xy_record entries), wolff_set_schedule (CLUSTER only),
 * wolff_get_info, wolff_get_stats and ising_free; the Ising state and
 * measure entry points, wolff_run_host and the batched form return
 * WOLFF_EUNSUPPORTED for it. */
#define WOLFF_XY_ANGLE_BITS 15
typedef struct {
    uint32_t C;
    uint32_t levels;
    int64_t  E;     /* fixed-point bond sum after the flip */
    int64_t  Mx;    /* fixed-point magnetisation after the flip */
    int64_t  My;
} wolff_xy_record;

/* Bytes of device workspace an XY context of this shape needs (0 if
 * invalid): 32-bit site words, the cluster list, the cosine table. */
size_t wolff_xy_workspace_bytes(int dim, int L);

/* As ising_init, for the XY model; angle_bits in 1..15 (EINVAL otherwise). */
wolff_status xy_init(wolff_ctx **out, int dim, int L, int angle_bits, double J, double T,
                     uint64_t seed, void *d_workspace, size_t workspace_bytes, void *stream);

/* Incrementally tracked E, Mx, My and the last cluster size (outputs
 * nullable).  Synchronises; reports latched device errors. */
wolff_status xy_measure(wolff_ctx *ctx, int64_t *E, int64_t *Mx, int64_t *My,
                        uint64_t *last_C);

/* The same three sums by a full pass over the lattice.  Synchronises. */
wolff_status xy_measure_full(wolff_ctx *ctx, int64_t *E, int64_t *Mx, int64_t *My);

/* Checkpoint / restore of the angles (N uint16 entries) and the next update
 * index.  set_state rejects, with EINVAL, angles off the context's grid and
 * recomputes E, Mx, My.  Both synchronise. */
wolff_status xy_get_state(wolff_ctx *ctx, uint16_t *h_theta, uint64_t *t);
wolff_status xy_set_state(wolff_ctx *ctx, const uint16_t *h_theta, uint64_t t);

/* Enqueues n_updates single-cluster updates (t .. t+n-1), each: seed site,
 * level-synchronous growth with atomic claims and warp-aggregated appends to
 * the cluster list, boundary-bond energy change, unmark, record.
 * Paper: section 2, steps (i)-(iv) and the ic/in list (the update), section
 * 4, step (iii') (growth by parallel expansion of the wave-front spins), and
 * section 5, Tables 1-2, "+ measurement" column (E and M after every
 * update).  d_records
 * (nullable) receives n_updates wolff_record entries.  n_updates = 0 is a
 * no-op.  Asynchronous. */
wolff_status wolff_step(wolff_ctx *ctx, uint64_t n_updates, void *d_records);

/* Same as wolff_step but through host memory: if h_spins_in is non-NULL the
 * lattice (int8 +-1, N entries) is first uploaded and t set to t_in; the
 * records (n_updates entries, nullable) and the final lattice (nullable) are
 * copied back.  Synchronises the stream. */
wolff_status wolff_run_host(wolff_ctx *ctx, const int8_t *h_spins_in,
                            uint64_t t_in, uint64_t n_updates,
                            wolff_record *h_records, int8_t *h_spins_out);

/* Reads the incrementally tracked E_bond, M and the size of the last cluster
 * (0 before the first update).  Paper: section 2 (E and M of the
 * Hamiltonian) and section 5 (measured after each update).  Synchronises the stream; reports latched
 * device errors.  Any output pointer may be NULL. */
wolff_status measure(wolff_ctx *ctx, int64_t *E_bond, int64_t *M,
                     uint64_t *last_C);

/* Recomputes E_bond and M by a full pass over the lattice (the verification
 * path; section 2's definitions summed directly).  Synchronises. */
wolff_status measure_full(wolff_ctx *ctx, int64_t *E_bond, int64_t *M);

/* Checkpoint: copies the lattice out as int8 +-1 (N entries, h_spins) and the
 * next update index.  Synchronises. */
wolff_status wolff_get_state(wolff_ctx *ctx, int8_t *h_spins, uint64_t *t);

/* Restore: uploads an int8 +-1 lattice and sets the next update index; E_bond
 * and M are recomputed.  EINVAL (latched, reported here) if an entry is not
 * +-1.  Synchronises. */
wolff_status wolff_set_state(wolff_ctx *ctx, const int8_t *h_spins, uint64_t t);

/* Bit-packed state transfers (Ising contexts): the lattice as ceil(N / 32)
 * 32-bit words, bit (i mod 32) of word i / 32 set when site i is +1 (site
 * order as above; the unused high bits of the last word are ignored on input
 * and zero on output).  One bit per site moves 8x fewer bytes over the host
 * link than the int8 form; the device keeps one byte per site.  Otherwise as
 * wolff_set_state, wolff_get_state and wolff_run_host (every input is valid,
 * so no EINVAL for entries).  Potts and XY contexts: WOLFF_EUNSUPPORTED. */
wolff_status wolff_set_state_bits(wolff_ctx *ctx, const uint32_t *h_bits, uint64_t t);
wolff_status wolff_get_state_bits(wolff_ctx *ctx, uint32_t *h_bits, uint64_t *t);
wolff_status wolff_run_host_bits(wolff_ctx *ctx, const uint32_t *h_bits_in, uint64_t t_in,
                                 uint64_t n_updates, wolff_record *h_records,
                                 uint32_t *h_bits_out);

/* Chooses the schedule and the CTA shape of the growth kernels (0 = keep /
 * library default).  For PERSISTENT and GRAPH grid_blocks is the number of
 * CTAs (PERSISTENT caps it at what can be co-resident); for CLUSTER it is the
 * cluster size (1, 2, 4, 8 or 16; 16 needs a GPU that allows non-portable
 * cluster sizes); for TINY it must be 0 or 1.  block_threads: a multiple of
 * 32, at most 512 for PERSISTENT and CLUSTER, 1024 for GRAPH (TINY: see
 * above).  TINY on a Potts or XY context, or on a
 * lattice of more than WOLFF_TINY_MAX_SITES sites, is EUNSUPPORTED.  Results
 * do not depend on the choice. */
wolff_status wolff_set_schedule(wolff_ctx *ctx, int schedule, int grid_blocks,
                                int block_threads);

/* Persistent schedule: a level whose new wave front exceeds t_up sites is
 * expanded by all CTAs (grid barrier per level) until a level produces at
 * most t_down sites, which CTA 0 then expands alone (__syncthreads per
 * level).  t_up = 0 puts every level on the grid.  Requires
 * t_down <= t_up <= 2048.  Results do not depend on the values. */
wolff_status wolff_set_local_thresholds(wolff_ctx *ctx, uint32_t t_up, uint32_t t_down);

/* Cluster schedule and batched runs: window mode (on by default).  While the
 * recent clusters are small, all warps of the team grow consecutive updates
 * speculatively on the current lattice, one update per warp at a time, each
 * taking the next free update of a window of up to 2048 when done.  Rounds
 * of `levels` growth levels alternate with commits: the prefix of finished
 * updates none of whose members, nor neighbours across open bonds, an
 * earlier one flips is applied in order, each boundary sum corrected for the
 * earlier flips of neighbours across closed bonds; an uncommitted update that
 * read a committed flip is grown again.  A committed update is exactly the
 * serial one (section 2's cluster depends only on those spins and on the
 * counter-based bond draws), so results do not depend on the setting.  enable: 0 = off, 1 = on with the default
 * levels per round (24 in 2D, 28 in 3D), k >= 2 = on with k levels per round
 * (at most 64).  EINVAL if enable < 0. */
wolff_status wolff_set_burst(wolff_ctx *ctx, int enable);

/* Helper teams (cluster schedule, window mode on, lattices of 2^20 sites or
 * more): a wolff_step launches, beside the cluster that runs the chain, as
 * many more clusters of the same shape as the GPU holds at once.  They grow
 * the launch's next updates ahead of it, on the lattice as they read it, into
 * the workspace's ring; the main cluster takes such a result only if every
 * spin its growth read -- the members, and each member's neighbours -- still
 * has the value the growth saw, in which case it is the cluster the main
 * cluster would grow itself (section 2's cluster depends only on those spins
 * and on the counter-based bond draws); otherwise it grows the update.  The
 * main cluster never waits for a helper, and results do not depend on the
 * setting.  max_helpers: -1 = as many as fit (the default), 0 = none,
 * k > 0 = at most k.  EINVAL if max_helpers < -1. */
wolff_status wolff_set_helpers(wolff_ctx *ctx, int max_helpers);

wolff_status wolff_get_info(wolff_ctx *ctx, wolff_info *info);

/* Counters of the persistent and cluster schedules, accumulated since
 * ising_init or the last wolff_set_state (tracing aid; the leader CTA's
 * thread 0 keeps them; in the cluster schedule "grid" means "cluster"). */
typedef struct {
    uint64_t updates;
    uint64_t levels_local;     /* levels grown by the leader CTA alone */
    uint64_t levels_grid;      /* levels grown by all CTAs */
    uint64_t ns_local;         /* device time (globaltimer) in leader-only growth */
    uint64_t ns_grid;          /* device time in all-CTA growth phases */
    uint64_t ns_finish;        /* device time closing updates (energy, unmark, record) */
    uint64_t handoffs;         /* leader -> all-CTA hand-offs */
    uint64_t grid_finishes;    /* updates closed by all CTAs */
    uint64_t start_ns;         /* device globaltimer when the last launch began this lattice */
    uint64_t end_ns;           /* ... and when it finished it */
    uint64_t burst_updates;    /* updates committed by window mode (cluster schedule) */
    uint64_t bursts;           /* window-mode commit rounds */
    uint64_t ns_win_grow;      /* window mode, leader's view: growth phases */
    uint64_t ns_win_map;       /*   flattening and recording the flips */
    uint64_t ns_win_check;     /*   conflict checks and the cut */
    uint64_t ns_win_commit;    /*   commits, records, regrowth queue */
    uint64_t win_levels;       /* growth levels run by all warps, discarded ones included */
    uint64_t pregrown;         /* window updates taken from the helper teams' ring */
    uint64_t ns_win_first_grow; /* growth phase of each window's first round (leader's view) */
    uint64_t win_regrown;      /* window updates grown again after a commit changed what they read */
    uint64_t win_fresh_grown;  /* fresh window updates the main team grew itself */
} wolff_stats;

/* Reads the counters above.  Synchronises. */
wolff_status wolff_get_stats(wolff_ctx *ctx, wolff_stats *stats);

/* Host-side Philox threshold the library uses for (J, T). */
uint64_t wolff_bond_threshold(double J, double T);

/* Fills d_out[4k .. 4k+3] with Philox4x32-10(key, d_ctr[4k .. 4k+3]) for k <
 * n on the device (test hook for the generator).  Asynchronous on stream. */
wolff_status wolff_philox(uint32_t key0, uint32_t key1, const uint32_t *d_ctr,
                          uint32_t *d_out, uint64_t n, void *stream);

/* Failure-detection self test: runs the library's bounded device-side wait
 * on a private control block where nothing can release it, with a limit of
 * wait_ns nanoseconds (<= 10 s).  *observed receives the status the device
 * latched: WOLFF_ETIMEOUT when the limit works.  The context's own state is
 * not touched and stays usable.  Synchronises. */
wolff_status wolff_selftest_wait_timeout(wolff_ctx *ctx, uint64_t wait_ns, int *observed);

/* ---- an update path that allocates nothing ------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc where they run updates: code inside a framework
 * whose caching allocator already owns the device memory, loops that cannot
 * afford cudaMalloc's implicit device-wide synchronisation, and programs that
 * fix their device-memory budget when the library is loaded.
 *
 * wolff_step_static runs n_updates updates (t0 .. t0+n-1, the same Philox
 * streams and results as a context with this dim, L, J, T and seed) on a
 * caller-owned lattice, using no workspace and allocating nothing.  Its
 * scratch (a 1 KiB control block and a cluster list of
 * WOLFF_STATIC_MAX_SITES 32-bit entries, 4 MiB + 1 KiB in all) is a
 * file-scope __device__ array, which every GPU that loads the library holds
 * until the process exits.
 *   d_spins    device int8 lattice of +-1 values (N = L^dim entries, site
 *              i = x + L*y (+ L*L*z)), 16-byte aligned, with room for
 *              N rounded up to a multiple of 4 bytes; updated in place;
 *   d_records  nullable, n_updates wolff_record entries, 8-byte aligned;
 *   stream     cudaStream_t (NULL = default stream); asynchronous.
 * Returns, before touching the lattice, WOLFF_EINVAL for a bad
 * shape/parameter, a misaligned lattice or record buffer, or
 * L^dim > WOLFF_STATIC_MAX_SITES, and WOLFF_ECUDA when a query of the
 * device fails.  WOLFF_ECUDA from a later launch still leaves the lattice
 * converted back to +-1.
 * Errors found on the device are latched in the static control block and
 * read by wolff_step_static_status (below), not by this call's return
 * value:
 *   - an entry other than +-1 latches WOLFF_EINVAL; no update runs, no
 *     record is written, and that entry comes back as -1;
 *   - a bounded wait that ran out latches WOLFF_ETIMEOUT; the updates stop
 *     at the next check (every 32 updates) and only the records of the
 *     completed updates are written.
 * Each call looks up the array's device address on the current device; the
 * first call on a device also loads the library's device code, so make it
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents (each call clears what must start at zero, its
 * status included), so calls whose work overlaps on the GPU -- on different
 * streams, or from different threads -- race and must be serialised by the
 * caller. */
#define WOLFF_STATIC_MAX_SITES (1u << 20)
wolff_status wolff_step_static(int dim, int L, double J, double T, uint64_t seed,
                               uint64_t t0, uint64_t n_updates, void *d_spins,
                               void *d_records, void *stream);

/* Synchronises `stream` (the one the last wolff_step_static call used) and
 * reads what that call's work latched on the device: *device_status = 0 or
 * a wolff_status (WOLFF_EINVAL, WOLFF_ETIMEOUT), *detail = where it was
 * raised (for EINVAL, the index of a bad entry), *t_next = the index
 * of the next update (t0 + the updates completed).  Outputs are nullable.
 * The next wolff_step_static call clears these values, so read them before
 * it.  Allocates nothing.  Returns WOLFF_ECUDA if the copy or the
 * synchronisation fails, else WOLFF_OK. */
wolff_status wolff_step_static_status(void *stream, int *device_status, uint32_t *detail,
                                      uint64_t *t_next);

/* ---- batched form: many lattices in one launch ----------------------------
 * A batch runs the next updates of several contexts in one kernel launch,
 * one thread-block cluster per context (the CLUSTER schedule's engine), so
 * hundreds of small lattices share the GPU instead of running one lattice per
 * launch.  Every context keeps its own chain: the results are those of
 * wolff_step on each context alone.  The batch owns a small descriptor table
 * on the device and a pinned host staging copy of it. */
typedef struct wolff_batch wolff_batch;

/* capacity: most contexts one wolff_batch_run may take; stream: where the
 * batched launches go (NULL = default stream). */
wolff_status wolff_batch_create(wolff_batch **out, int capacity, void *stream);

/* Enqueues n_updates[i] updates of ctxs[i] for i < n (0 skips a context),
 * records to d_records[i] (nullable entries).  The contexts must be distinct,
 * live on the batch's device, and have no work pending on other streams.
 * Larger lattices are launched first.  cluster_size (1..16) and
 * block_threads (multiple of 32, <= 512) set the team shape (a TINY batch:
 * see wolff_batch_set_schedule).  Asynchronous
 * on the batch's stream; device errors are reported by each context's next
 * synchronising call. */
wolff_status wolff_batch_run(wolff_batch *b, wolff_ctx *const *ctxs, int n,
                             const uint64_t *n_updates, void *const *d_records,
                             int cluster_size, int block_threads);

/* As wolff_batch_run, but every lattice stops at the first update boundary
 * after budget_ns nanoseconds of device time from the start of its work
 * (0 = no limit), so a lattice whose updates suddenly get dearer cannot hold
 * a batch for long.  How many updates each lattice ran is known after the
 * next synchronising call on its context (wolff_get_stats().updates,
 * wolff_get_info().t); its records fill a prefix of d_records[i]. */
wolff_status wolff_batch_run_timed(wolff_batch *b, wolff_ctx *const *ctxs, int n,
                                   const uint64_t *n_updates, void *const *d_records,
                                   int cluster_size, int block_threads, uint64_t budget_ns);

/* Window slots per CTA of this batch's launches (window mode's queue of
 * speculative updates, see wolff_set_burst): 16, 32, 64 (the default) or
 * 128, or 0 to run the batch without window mode.  Larger windows hold more
 * updates in flight and need more shared memory; a team shape whose window
 * does not fit makes the next wolff_batch_run fail with WOLFF_ECUDA.  The
 * levels per round come from each context's wolff_set_burst.  Results do not
 * depend on the setting.  EINVAL for other values. */
wolff_status wolff_batch_set_window(wolff_batch *b, int slots_per_cta);

/* The engine of this batch's launches: WOLFF_SCHED_CLUSTER (the default: one
 * thread-block cluster per context, window mode) or WOLFF_SCHED_TINY (one
 * CTA per context holding its lattice in shared memory as bit planes, see
 * the TINY schedule; one launch per dimension).  On a TINY batch every
 * context must be an Ising lattice of at most WOLFF_TINY_MAX_SITES sites
 * (wolff_batch_run: EUNSUPPORTED otherwise), cluster_size must be 1, and
 * block_threads is 0 (each launch takes TINY's default for its largest
 * lattice) or a CTA size that lattice can use (EINVAL otherwise).  Results
 * do not depend on the engine.  EINVAL for other values. */
wolff_status wolff_batch_set_schedule(wolff_batch *b, int schedule);

wolff_status wolff_batch_free(wolff_batch *b);

/* ---- measurement aid ------------------------------------------------------
 * L2 bandwidth probe (the paper has no counterpart; it gives the L2 side of
 * the growth kernels' memory roofline, whose working set lives in L2).
 * Streams the device buffer d_buf (`bytes` bytes, a multiple of 16, 16-byte
 * aligned) `passes` times (1..100000) in one launch of a full-occupancy grid
 * over all SMs, with 16-byte loads that skip L1; mode 0 only reads, mode 1
 * also writes every vector back (its contents change).  d_sink: one
 * 4-byte-aligned device word the kernel may write (so its loads stay live).
 * With `bytes` well inside L2, every pass after the first is served by L2:
 * passes * bytes (mode 1: twice that) over the launch's CUDA-event time is
 * the L2 bandwidth.  EINVAL for bad arguments, ECUDA if a device query or the
 * launch fails.  Asynchronous on stream (NULL = default stream). */
wolff_status wolff_l2_probe(void *d_buf, size_t bytes, int passes, int mode, uint32_t *d_sink,
                            void *stream);

/* Releases the context (and the workspace if the library allocated it).
 * Synchronises the stream first. */
wolff_status ising_free(wolff_ctx *ctx);

/* Last error message of the context (never NULL; "" if none). */
const char *wolff_last_error(wolff_ctx *ctx);

const char *wolff_status_string(wolff_status s);

#ifdef __cplusplus
}
#endif

#endif /* WOLFF_H */
