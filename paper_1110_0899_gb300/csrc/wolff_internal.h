// wolff_internal.h -- structures shared by the library's host and device code.
//
// Device memory of one context (the caller's workspace), 256-byte aligned
// pieces:
//   [DevCtl][self-test DevCtl][spins: N bytes, padded to 256][list: N x u32]
// spins: one byte per site, bit 0 = current spin, bit 1 = spin at the start
//   of the running update (+1 stored as 1).  Between updates the two bits are
//   equal, so a byte is 0x00 (-1) or 0x03 (+1).  Claiming a site flips bit 0
//   only; a cluster member is a site whose two bits differ.
// list: the cluster list of section 2 (ic = members, in = checked); entries
//   are packed lattice coordinates (2D: x | y << 16, 3D: x | y << 10 | z << 20)
//   so that no division is needed to find neighbours.  Level k's frontier is a
//   contiguous range of it.
#pragma once

#include <stdint.h>

#include "wolff.h"

namespace wolff {

constexpr uint32_t kTagBond = 0;
constexpr uint32_t kTagSeed = 1;
constexpr uint32_t kTagInit = 2;

// Value of an empty cluster-list slot.  Every slot holds it between updates
// (the unmark pass restores it), so a reader that finds anything else in a
// slot of the running update is looking at that update's entry: list entries
// need no release/acquire ordering, only the level counts do.  Packed
// coordinates never take this value (2D coordinates are < 2^15, 3D < 2^10).
constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;

// Control block living at the start of the workspace.  Fields are grouped
// into 128-byte lines by who touches them: the chain state (one thread at a
// time), the grid barrier, the leader's command word, the append counters and
// the graph schedule's state.
struct alignas(256) DevCtl {
    // line 0: chain state
    unsigned long long t;          // next update index
    long long E;                   // bond sum
    long long M;                   // magnetisation
    unsigned long long total_C;    // sum of cluster sizes so far
    unsigned int last_C;
    unsigned int last_levels;
    unsigned int status;           // 0 or a wolff_status (atomic, first wins)
    unsigned int err_detail;       // where a bounded wait gave up, etc.
    long long full_E;              // full recount results
    long long full_M;
    long long My;                  // XY: second magnetisation component
    long long full_My;
    unsigned int up_blocks;        // blocks of the fused upload pass done (atomic)
    // line 1: grid barrier
    // bar_word = arrivals << 32 | entries appended this level (atomic): the
    // warps reserve list slots and the CTAs arrive on the same word, so the
    // last arrival knows the level's total without another round trip.
    // bar_pub = generation << 32 | that total, published with a release store.
    alignas(128) unsigned long long bar_word;
    unsigned long long bar_pub;
    // line 2: leader -> worker commands
    alignas(128) unsigned int cmd_seq;
    unsigned int cmd_kind;
    unsigned int cmd_lo, cmd_hi, cmd_level, cmd_sig0bit;
    unsigned long long cmd_t;
    unsigned long long cmd_rec;            // record index of the update
    // line 3: append counters and the boundary-bond sum
    alignas(128) unsigned int cnt[4];      // (atomic)
    long long dE;                          // (atomic)
    // line 4: graph schedule state
    alignas(128) unsigned int lo, hi;      // current frontier = list[lo, hi)
    unsigned int levels;
    unsigned int done;                     // CTAs finished in this kernel (atomic)
    unsigned int sig0bit;                  // seed spin (1 = +1) of the running update
    unsigned int pad0;
    unsigned long long t_end;              // graph loop stops when t == t_end
    unsigned long long rec_t0;             // t of records[0] for this call
    wolff_record *records;                 // destination of this call's records
    // line 5: persistent-schedule counters (leader thread, accumulated)
    alignas(128) unsigned long long st_updates;
    unsigned long long st_levels_local, st_levels_grid;
    unsigned long long st_ns_local, st_ns_grid, st_ns_finish;
    unsigned long long st_handoffs, st_grid_finishes;
    unsigned long long st_start_ns, st_end_ns;   // globaltimer at the last launch's start/end
    unsigned long long st_burst_updates;         // updates committed by window mode
    unsigned long long st_bursts;                // window-mode commit rounds
    // line 6: window-mode phase times (leader thread 0) and growth work
    alignas(128) unsigned long long st_ns_win[4];   // growth, map, check, commit
    unsigned long long st_win_levels;            // growth levels of all warps (incl. discarded)
    unsigned long long st_pregrown;              // window updates taken pre-grown from the ring
    unsigned long long st_ns_win_first;          // growth phase of each window's first round
    unsigned long long st_win_regrown;           // window updates grown again (regrowth queue)
    unsigned long long st_win_fresh_grown;       // fresh window updates the main team grew itself
    // the pre-growing helper teams of a one-lattice launch, per launch parity
    // (launch epoch & 1; a launch clears the other parity's words for the
    // next one, which cannot start before it has ended)
    unsigned int pg_next[2];                     // next update to pre-grow (atomic)
    unsigned int pg_stop[2];                     // the launch's main team has finished
    unsigned int pg_commit[2];                   // updates of the launch committed so far
    unsigned int pg_done[2];                     // results the helpers have written (atomic)
};
static_assert(sizeof(DevCtl) % 256 == 0 && sizeof(DevCtl) <= 1024, "control block layout");

struct Geometry {
    uint32_t L;
    uint32_t N;
    uint32_t LL;         // L*L
};

struct StepParams {
    uint8_t *spins;
    uint32_t *list;
    DevCtl *ctl;
    wolff_record *records;      // nullable
    Geometry g;
    uint32_t key0, key1;
    unsigned long long thr;     // 0 .. 2^32
    unsigned long long t0;      // first update of this launch
    unsigned long long n;       // updates in this launch
    unsigned long long wait_ns; // bound of every device-side wait
    uint32_t t_up;              // leader hands a frontier larger than this to the grid
    uint32_t t_down;            // grid hands a frontier this small back to the leader
    uint32_t win_levels;        // cluster schedule: window mode, growth levels per round (0 = off)
    unsigned long long budget_ns;   // cluster schedule: stop after this much device time (0 = none)
    uint32_t q;                 // Potts: number of colours (the Ising kernels ignore it)
    // XY (the other kernels ignore these): the sites are 32-bit words
    // (angle | claim bit), spins points at them
    const int32_t *xy_tab;      // fixed-point quarter-wave cosine table, 16385 entries
    const double *xy_coef;      // 1/n!, n = 0..16, for e^-y
    double xy_kk;               // 2 J / T * 2^-60
    uint32_t xy_bits;           // angle grid: spins multiples of 2^(16-bits)
    wolff_xy_record *xy_records;
    // pre-grown updates (one-lattice cluster launches with helper teams):
    // ring of kRingSlots slots of kRingSlotBytes, nullable
    uint8_t *ring;
    uint32_t pg_epoch;          // launch counter of the context (its parity selects the words)
    uint32_t pg_lead;           // helpers grow update u only once u < committed + pg_lead
    unsigned long long pg_wait_ns;  // main team: longest wait for the helpers' first window
};

// The ring of pre-grown updates: update u of a launch (counted from the
// launch's first update) goes to slot u mod kRingSlots.  A slot holds
//   [0, 8)     tag: the launch's epoch << 32 | (u + 1), written last (release);
//              the ring is zeroed when its context is created, so a tag is
//              unique among the context's own launches
//   [16, 32)   uint4 (|C|, levels, dE_bond / 2, seed spin); |C| = 0 marks an
//              update too big to pre-grow
//   [32, ...)  the members (packed coordinates, up to 128), then the three
//              per-member bond masks of window mode (alignment, open, boundary),
//              128 bytes each.
constexpr uint32_t kRingSlots = 4096;
constexpr uint32_t kRingSlotBytes = 1024;
constexpr uint32_t kRingMembersOff = 32;
constexpr uint32_t kRingMaxCap = 128;
constexpr uint32_t kRingMasksOff = kRingMembersOff + 4 * kRingMaxCap;
static_assert(kRingMasksOff + 3 * kRingMaxCap <= kRingSlotBytes, "ring slot layout");
// lattices of at least this many sites get a ring (and helper teams)
constexpr uint32_t kRingMinSites = 1u << 20;

// Leader-local frontier capacity (shared memory) and the cluster-list prefix
// kept in shared memory for the leader-only energy/unmark pass.
constexpr uint32_t kLocalFrontierCap = 2048;
constexpr uint32_t kLocalListCap = 4096;

// Launch helpers implemented in wolff_kernels.cu (C++ linkage, internal).
cudaError_t launch_init(uint8_t *spins, Geometry g, uint32_t k0, uint32_t k1,
                        cudaStream_t s);
cudaError_t launch_measure_full(int dim, const uint8_t *spins, Geometry g,
                                DevCtl *ctl, int set_chain, cudaStream_t s);
cudaError_t launch_from_pm1(uint8_t *spins, const int8_t *src, uint32_t N,
                            DevCtl *ctl, cudaStream_t s);
cudaError_t launch_from_pm1_measure(int dim, uint8_t *spins, const int8_t *src, Geometry g,
                                    DevCtl *ctl, cudaStream_t s);
cudaError_t launch_from_bits_measure(int dim, uint8_t *spins, const uint32_t *bits, Geometry g,
                                     DevCtl *ctl, cudaStream_t s);
cudaError_t launch_to_bits(uint32_t *bits, const uint8_t *spins, uint32_t N, cudaStream_t s);
cudaError_t launch_to_pm1(int8_t *dst, const uint8_t *spins, uint32_t N,
                          cudaStream_t s);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr,
                          uint32_t *out, unsigned long long n, cudaStream_t s);
cudaError_t launch_reset_ctl(DevCtl *ctl, unsigned long long t, cudaStream_t s);
cudaError_t launch_prelaunch(DevCtl *ctl, cudaStream_t s);
cudaError_t launch_prefetch_l2(const void *base, unsigned long long bytes, cudaStream_t s);

// Persistent cooperative schedule.
const void *persistent_kernel(int dim);
int persistent_max_blocks_per_sm(int dim, int threads, int *err);

// Team schedule (wolff_team.cu): one thread-block cluster per job; the jobs
// come from d_table (device array of njobs StepParams) or, when d_table is
// null, the single job `single` (njobs must be 1).
// Window mode (speculative growth of many small updates at once) needs
// window_slots (a power of two, 0 = off) slots per CTA of dynamic shared memory.
struct WinCfg {
    uint32_t slots;   // window slots per CTA (0: no window area, window mode off)
    uint32_t cap;     // members per speculative update
    uint32_t helpers; // one-lattice launches: clusters after the first that pre-grow
                      // updates into the ring (0 = none)
};
// Growth levels per warp between commit rounds, by dimension: the fastest of
// 12, 16, 20, 24, 28, 32 and 48 on the 2D L=4096 and 3D L=256 random-start
// chains in 10^4-update launches.
inline int default_window_levels(int dim) { return dim == 3 ? 28 : 24; }
const void *team_kernel(int dim);
// Raises the team kernel's dynamic shared-memory limit to at least `bytes`
// (on the current device); never lowers it.
cudaError_t ensure_team_dyn_smem(int dim, size_t bytes);
uint32_t window_cap(int dim, int threads);
size_t window_smem_bytes(int dim, int threads, int window_slots, int cluster_size);
cudaError_t launch_team(int dim, const StepParams &single, const StepParams *d_table, int njobs,
                        int cluster_size, int threads, int window_slots, cudaStream_t s,
                        int helpers = 0);
// Clusters of this shape that can be resident at once (0 if the query fails).
int team_max_active_clusters(int dim, int cluster_size, int threads, int window_slots);

// q-state Potts (wolff_potts.cu).
cudaError_t launch_potts_init(uint8_t *spins, Geometry g, uint32_t q, uint32_t k0, uint32_t k1,
                              cudaStream_t s);
cudaError_t launch_potts_measure(int dim, const uint8_t *spins, Geometry g, DevCtl *ctl,
                                 int set_chain, cudaStream_t s);
cudaError_t launch_potts_check(const uint8_t *spins, uint32_t N, uint32_t q, DevCtl *ctl,
                               cudaStream_t s);
cudaError_t launch_potts_team(int dim, const StepParams &p, int cluster_size, int threads,
                              cudaStream_t s);

// XY embedded-cluster model (wolff_xy.cu).
constexpr uint32_t kXyTableSize = 16385;
cudaError_t launch_xy_init(uint32_t *words, Geometry g, uint32_t bits, uint32_t k0, uint32_t k1,
                           cudaStream_t s);
cudaError_t launch_xy_measure(int dim, const uint32_t *words, Geometry g, const int32_t *tab,
                              DevCtl *ctl, int set_chain, cudaStream_t s);
cudaError_t launch_xy_check(const uint32_t *words, uint32_t N, uint32_t bits, DevCtl *ctl,
                            cudaStream_t s);
cudaError_t launch_xy_team(int dim, const StepParams &p, int cluster_size, int threads,
                           cudaStream_t s);

// Graph schedule: builds the nested-WHILE graph; returns its executable.
cudaError_t build_update_graph(int dim, const StepParams &p, int blocks,
                               int threads, cudaGraphExec_t *exec,
                               cudaGraph_t *graph);
cudaError_t launch_graph_call(DevCtl *ctl, unsigned long long n,
                              wolff_record *records, cudaStream_t s);

}  // namespace wolff
