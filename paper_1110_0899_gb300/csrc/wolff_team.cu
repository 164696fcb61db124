// wolff_team.cu -- the Wolff update run by a thread-block cluster ("team").
//
// One cluster of CS CTAs owns one lattice (a job) for the whole launch and
// runs its n updates.  Clusters never wait on one another, so a launch may
// hold any number of jobs -- one lattice (the plain form) or hundreds of
// independent replicas (the batched form) -- and the hardware schedules the
// clusters as SMs free up.  Inside a team:
//   - rank 0 (the leader) grows small wave fronts alone, with __syncthreads
//     as the level barrier and the front in shared memory (the on-GPU form of
//     the paper's hybrid, section 6);
//   - a front above t_up is expanded by all CTAs of the cluster, each taking
//     a stride of list[lo, hi); new sites get their list slots from counters
//     in the leader's shared memory (distributed shared memory atomics) and
//     levels are separated by the cluster barrier (barrier.cluster, release/
//     acquire at cluster scope), the GB300 hardware replacement of the
//     paper's quasi-block synchronisation (section 3).
// The worker CTAs of a team block in the cluster barrier while the leader
// works alone; every CTA of a cluster executes the same sequence of cluster
// barriers (the leader announces each team phase in its shared memory before
// the barrier that starts it), so the hardware barrier always completes.  The
// workers read the leader's shared memory remotely, so the team leaves the
// kernel only after a last cluster barrier that follows every such read.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>

#include "wolff_device.cuh"

namespace cg = cooperative_groups;

namespace wolff {

namespace {

enum : unsigned int { kTeamLevels = 1, kTeamFinish = 2, kTeamExit = 3, kTeamWindow = 4 };

// ---- window mode -------------------------------------------------------------
// While clusters are small, consecutive updates rarely touch the same sites.
// Window mode then grows many consecutive updates at once, all on the current
// lattice, without claiming anything: each warp grows one update at a time
// (its cluster in a shared-memory hash set) and, when done, takes the next
// free update of its CTA.  The window holds updates [c, c + P), P = S slots
// per CTA times the cluster size; update j lives in CTA j mod CS, slot
// (j / CS) mod S.  Rounds of K levels of growth alternate with commits:
//   - every finished update records the sites it flips in a map "lowest
//     update index that flips this site": the cluster-list array indexed by
//     site, written with L2 atomics and read with L2 loads;
//   - update j conflicts if an earlier finished update of the window flips
//     one of its members or a neighbour across an open boundary bond (draw
//     below the threshold): only those flips can change its cluster;
//   - the round commits [c, cut), cut = the first update that is unfinished
//     or conflicts: it flips their members and writes their records, each
//     boundary sum corrected for the earlier flips of neighbours across
//     closed bonds (a closed bond's neighbour stays out whatever its spin,
//     and its term only changes sign);
//   - every uncommitted update, finished or still growing, that read a site
//     the committed ones flip is grown again from its seed; the others keep
//     their clusters, which the new lattice leaves unchanged.
// A committed update therefore finds the component, level count, boundary
// sum and record of the serial chain.  An update whose cluster outgrows the
// cap (or whose flips do not fit the map) stops the window; it runs the
// ordinary way.
constexpr int kWinMaxWarps = 16;
constexpr uint32_t kWinCap = 64;            // members per speculative update (see window_cap)
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kWinMaxStall = 4096;     // rounds without a commit before giving up
// Windows that commit fewer than kWinLowYield updates per round are left for
// the ordinary path, with the longest back-off: judged over kWinLowRounds
// rounds in a row within one call, and over the rounds of all windows since
// the last back-off (halved every 64 rounds, so that recent ones weigh most)
// once those reach kWinLowRounds.  This is the regime of small lattices near
// T_c, where nearly every update conflicts with the one before it and most
// windows soon stop at an update too big for them.
constexpr uint32_t kWinLowYield = 2;
constexpr uint32_t kWinLowRounds = 8;
enum : uint32_t { kSlotFree = 0, kSlotGrowing = 1, kSlotDone = 2, kSlotTooBig = 3, kSlotRegrow = 4 };

struct TeamShared {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];        // level append counters (the leader's are the team's)
    unsigned int sig0bit;
    unsigned int cmd[8];        // kind, lo, hi, level, sig0bit, t_lo, t_hi
    unsigned long long dE;      // team boundary sum (leader's copy)
    // window mode (the leader's copies are the team's)
    unsigned int wcut;          // lowest update of the window that cannot commit (atomic)
    unsigned int wlimit;        // lowest update found too big (atomic)
    unsigned int wstop;         // time budget spent
    unsigned int wflag;         // leader: this update starts (or resumes) a window
    unsigned int wlowy;         // leader: the last window was left for committing too little
    unsigned int budget_stop;   // leader: the time budget stops the launch here
    unsigned int wlast[2];      // |C| and levels of the last committed update
    unsigned long long wlevels; // growth levels of all warps (atomic)
    long long wsum[3][kWinMaxWarps];  // per-warp totals of the record scan
    long long wbase[3];         // E_bond, M and sum of |C| before the scanned block
};

// All CTAs of the team: expand level after level from list[lo, hi) until the
// next front is empty (*finished) or has t_down sites or fewer.
template <int DIM>
__device__ __forceinline__ void team_levels(const StepParams &p, TeamShared &sh,
                                            cg::cluster_group &cl, uint32_t &lo, uint32_t &hi,
                                            uint32_t &level, uint32_t sig0bit, uint32_t tlo,
                                            uint32_t thi, bool *finished) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t gw = rank * warps + warp, nw = cs * warps;
    while (true) {
        unsigned int *cnt = &lead->cnt[level % 3];
        if (rank == 0 && threadIdx.x == 0) sh.cnt[(level + 1) % 3] = 0;
        for (uint32_t b = lo + gw * 32u; b < hi; b += nw * 32u) {
            const uint32_t k = b + lane;
            Neighbours<DIM> nb;
            uint32_t won = 0;
            if (k < hi) won = expand_site<DIM>(p, __ldcg(p.list + k), sig0bit, tlo, thi, nb);
            uint32_t pos = hi + warp_reserve(cnt, __popc(won));
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) {
                if (won & (1u << s)) {
                    if (pos < p.g.N) p.list[pos] = nb.packed[s];
                    else raise_status(p.ctl, WOLFF_EINVAL, 0xD0u);
                    ++pos;
                }
            }
        }
        cl.sync();
        uint32_t added = *reinterpret_cast<volatile unsigned int *>(cnt);
        ++level;
        if (added > p.g.N - hi) {   // cannot happen: every site joins at most once
            if (rank == 0 && threadIdx.x == 0) raise_status(p.ctl, WOLFF_EINVAL, 0xD1u);
            added = 0;
        }
        lo = hi;
        hi += added;
        if (added == 0 || added <= p.t_down) {
            *finished = added == 0;
            // every CTA has read the count before the leader reuses the counters
            cl.sync();
            return;
        }
    }
}

// All CTAs of the team: boundary sum over list[0, C), then unmark.  Returns
// the sum in the leader's thread 0.
template <int DIM>
__device__ __forceinline__ long long team_finish(const StepParams &p, TeamShared &sh,
                                                 cg::cluster_group &cl, uint32_t C,
                                                 uint32_t sig0bit) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t tid = rank * blockDim.x + threadIdx.x, nt = cs * blockDim.x;
    long long acc = 0;
    for (uint32_t k = tid; k < C; k += nt) {
        uint32_t i;
        acc += boundary_term<DIM>(p, __ldcg(p.list + k), sig0bit, &i);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0 && acc != 0) atomicAdd(&lead->dE, (unsigned long long)acc);
    cl.sync();
    long long dE = 0;
    if (rank == 0 && threadIdx.x == 0) {
        dE = (long long)sh.dE;
        sh.dE = 0;
    }
    for (uint32_t k = tid; k < C; k += nt) {
        uint32_t c[DIM];
        unpack<DIM>(__ldcg(p.list + k), c);
        unmark_site(p.spins, site_index<DIM>(p.g, c), sig0bit);
        p.list[k] = kEmptySlot;
    }
    cl.sync();
    return dE;
}

template <int DIM>
__device__ uint32_t team_window(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                                const WinCfg &wc, unsigned long long u0, uint32_t n_rem,
                                unsigned long long launch_t0, long long &E, long long &M,
                                unsigned long long &total_C, uint32_t &last_C,
                                uint32_t &last_levels, unsigned long long &rounds,
                                unsigned long long *win_ns, uint32_t c_start, bool resume,
                                bool &resumable);

template <int DIM>
__device__ void team_worker(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                            const WinCfg &wc) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    while (true) {
        cl.sync();   // the leader has announced the next phase
        const volatile unsigned int *cmd = lead->cmd;
        const unsigned int kind = cmd[0];
        uint32_t lo = cmd[1], hi = cmd[2], level = cmd[3];
        const uint32_t sig0bit = cmd[4], tlo = cmd[5], thi = cmd[6];
        if (kind == kTeamLevels) {
            bool finished = false;
            team_levels<DIM>(p, sh, cl, lo, hi, level, sig0bit, tlo, thi, &finished);
        } else if (kind == kTeamFinish) {
            team_finish<DIM>(p, sh, cl, hi, sig0bit);
        } else if (kind == kTeamWindow) {
            long long E = 0, M = 0;
            unsigned long long tc = 0, rounds = 0;
            uint32_t lc = 0, ll = 0;
            bool resumable = false;
            team_window<DIM>(p, sh, cl, wc, ((unsigned long long)hi << 32) | lo, level, 0, E, M,
                             tc, lc, ll, rounds, nullptr, tlo, sig0bit != 0, resumable);
        } else {
            // the leader's shared memory (read above) must outlive every
            // remote access: leave together, after one more cluster barrier
            cl.sync();
            return;
        }
    }
}

// ---- the warps' cluster hash sets --------------------------------------------
// Multiplicative (Fibonacci) hashing: the top log2(slots) bits of key * 2^32/phi.
__device__ __forceinline__ uint32_t set_hash(uint32_t key, uint32_t slots) {
    return (key * 0x9E3779B1u) >> (32 - __ffs(slots) + 1);
}

// Inserts key into an open-addressing set of `slots` entries (power of two).
// Returns 1 if newly inserted, 0 if present, -1 if the set is full.
__device__ __forceinline__ int set_insert(uint32_t *set, uint32_t slots, uint32_t key) {
    uint32_t h = set_hash(key, slots);
    for (uint32_t probe = 0; probe < slots; ++probe) {
        const uint32_t prev = atomicCAS(set + h, kEmptyKey, key);
        if (prev == kEmptyKey) return 1;
        if (prev == key) return 0;
        h = (h + 1) & (slots - 1);
    }
    return -1;
}

__device__ __forceinline__ bool set_contains(const uint32_t *set, uint32_t slots, uint32_t key) {
    uint32_t h = set_hash(key, slots);
    for (uint32_t probe = 0; probe < slots; ++probe) {
        const uint32_t v = set[h];
        if (v == key) return true;
        if (v == kEmptyKey) return false;
        h = (h + 1) & (slots - 1);
    }
    return false;
}

// The window's per-CTA state in dynamic shared memory: S slots of `cap`
// members (packed coordinates), each slot's result (|C|, levels, dE_bond / 2,
// seed spin) as one 16-byte word, then per slot the update index, state,
// lowest update it conflicts with, lowest update that flips any site it read,
// and the correction of its boundary sum; the regrowth queue, each slot's seed
// site, the slot offsets of the flattened member list and a few counters; and
// per member three bit masks over its 2 DIM bonds (bit s = bond to neighbour s):
//   amask: the neighbour was parallel to the seed spin when the growth read it
//          (also revalidates a finished update after a change of the lattice
//          made outside the window),
//   omask: the bond's draw is below the threshold (the bond is open),
//   bmask: the neighbour is not a member (a boundary bond).
struct WinView {
    uint32_t *members, *j, *state, *cmin, *amin, *rg, *seed, *off, *scal;
    int *dcorr;
    uint4 *meta;
    uint8_t *amask, *omask, *bmask;
    uint4 *lmeta;   // leader: results of updates c .. c + P - 1, pushed by their CTAs
};
enum : uint32_t { kScNextQ = 0, kScRgCount = 1, kScRgTake = 2, kScQEnd = 3, kScMin = 4,
                  kScSeeded = 5, kScSeedLo = 6 };
constexpr uint32_t kWinScalars = 8;

// Layout (32-bit words unless noted): members S*cap | meta S uint4 | lmeta
// S*cs uint4 | j, state, cmin, amin, dcorr, rg, seed S each | off S+1 | scalars |
// amask, omask, bmask S*cap bytes each.  Both uint4 arrays start at multiples
// of 16 bytes (cap is a multiple of 4 and the base is 16-byte aligned).
__device__ __forceinline__ WinView win_view(uint32_t *base, uint32_t S, uint32_t cap,
                                            uint32_t cs) {
    WinView v;
    v.members = base;
    v.meta = reinterpret_cast<uint4 *>(base + S * cap);
    v.lmeta = v.meta + S;
    uint32_t *m = base + S * cap + 4 * S + 4 * S * cs;
    v.j = m;
    v.state = m + S;
    v.cmin = m + 2 * S;
    v.amin = m + 3 * S;
    v.dcorr = reinterpret_cast<int *>(m + 4 * S);
    v.rg = m + 5 * S;
    v.seed = m + 6 * S;
    v.off = m + 7 * S;          // S + 1 entries
    v.scal = m + 8 * S + 1;     // kWinScalars
    v.amask = reinterpret_cast<uint8_t *>(m + 8 * S + 1 + kWinScalars);   // S * cap bytes
    v.omask = v.amask + S * cap;
    v.bmask = v.omask + S * cap;
    return v;
}

__device__ __forceinline__ void win_tick(unsigned long long &acc, unsigned long long &tick) {
    const unsigned long long now = global_ns();
    acc += now - tick;
    tick = now;
}

// Warp 0: off[s] = members of the finished slots before slot s, off[S] = all.
__device__ __forceinline__ void win_flatten(const WinView &v, uint32_t S, uint32_t lane) {
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 < S; k0 += 32) {
        const uint32_t s = k0 + lane;
        const uint32_t x = (s < S && v.state[s] == kSlotDone) ? v.meta[s].x : 0;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (s < S) v.off[s] = carry + incl - x;
        carry += __shfl_sync(kFullMask, incl, 31);
    }
    if (lane == 0) v.off[S] = carry;
}

// Warp 0: the regrowth queue, lowest update first (window starts at c).
__device__ __forceinline__ void win_queue(const WinView &v, uint32_t S, uint32_t c, uint32_t rank,
                                          uint32_t cs, uint32_t lane) {
    const uint32_t qlo = c > rank ? (c - rank + cs - 1) / cs : 0;
    uint32_t count = 0;
    for (uint32_t k0 = 0; k0 < S; k0 += 32) {
        const uint32_t s = (qlo + k0 + lane) & (S - 1);
        const bool want = k0 + lane < S && v.state[s] == kSlotRegrow;
        const uint32_t mask = __ballot_sync(kFullMask, want);
        if (want) v.rg[count + __popc(mask & ((1u << lane) - 1u))] = s;
        count += __popc(mask);
    }
    if (lane == 0) {
        v.scal[kScRgCount] = count;
        v.scal[kScRgTake] = 0;
    }
}

// Slot s holding update j of the flattened list entry f: off[s] <= f < off[s+1].
__device__ __forceinline__ uint32_t flat_slot(const uint32_t *off, uint32_t S, uint32_t f) {
    uint32_t lo = 0, hi = S;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= f) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void prefetch_l1(const void *ptr) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr));
}

// Lines a member j, added through direction s >= 2 (along y or z), reads
// when it expands that its parent's level did not: the next row (or plane)
// on along s, and in 3D the two lines beside j along the other of y, z.
// Indices are taken mod N; a wrong line at a wrap only costs a prefetch.
template <int DIM>
__device__ __forceinline__ void prefetch_two_hop(const Geometry &g, const uint8_t *spins,
                                                 uint32_t j, uint32_t s) {
    const uint32_t N = g.N;
    const uint32_t st = (s >> 1) == 1 ? g.L : g.LL;
    const uint32_t ahead = (s & 1u) ? (j >= st ? j - st : j + N - st)
                                    : (j + st < N ? j + st : j + st - N);
    prefetch_l1(spins + ahead);
    if (DIM == 3) {
        const uint32_t o = (s >> 1) == 1 ? g.LL : g.L;
        prefetch_l1(spins + (j + o < N ? j + o : j + o - N));
        prefetch_l1(spins + (j >= o ? j - o : j + N - o));
    }
}

// A spin read of the growth: through L1 for the main team, whose lattice
// changes only between its own cluster barriers; relaxed at GPU scope for a
// pre-growing helper, which reads the lattice while the main team commits.
template <bool kHelper>
__device__ __forceinline__ uint32_t grow_read(const uint8_t *p) {
    if constexpr (kHelper) return ld_relaxed_u8(p);
    else return (uint32_t)__ldca(p);
}

// Warp: a fresh speculative growth of the update with seed site i0 (claimed
// in the hash set).
template <int DIM, bool kHelper = false>
__device__ __forceinline__ void win_start(const StepParams &p, uint32_t i0, uint32_t *members,
                                          uint32_t *hset, uint32_t hslots, uint32_t lane,
                                          uint32_t &n, uint32_t &lo, uint32_t &levels,
                                          uint32_t &sig0bit) {
    for (uint32_t k = lane; k < hslots; k += 32) hset[k] = kEmptyKey;
    __syncwarp();
    sig0bit = grow_read<kHelper>(p.spins + i0) & 1u;
    // the first level reads the rows next to the seed's (index +-L, and +-L^2
    // in 3D, taken mod N: a wrong line at a wrap only costs a prefetch)
    if (!kHelper && lane < 2 * (DIM - 1)) {
        const uint32_t step = (lane >> 1) == 0 ? p.g.L : p.g.LL;
        const uint32_t N = p.g.N;
        const uint32_t nb = (lane & 1u) ? (i0 >= step ? i0 - step : i0 + N - step)
                                        : (i0 + step < N ? i0 + step : i0 + step - N);
        prefetch_l1(p.spins + nb);
    }
    if (lane == 0) {
        set_insert(hset, hslots, i0);
        members[0] = pack_index<DIM>(p.g, i0);
    }
    __syncwarp();
    n = 1;
    lo = 0;
    levels = 0;
}

// Neighbour s of the member `packed` (s = 2d: forward along axis d, 2d + 1:
// backward): its site index and packed coordinates, and the owner of the bond
// (the member for a forward bond, the neighbour for a backward one).
template <int DIM>
__device__ __forceinline__ void neighbour_of(const Geometry &g, uint32_t packed, uint32_t s,
                                             uint32_t &self, uint32_t &j, uint32_t &pj,
                                             uint32_t &owner) {
    uint32_t c[DIM];
    unpack<DIM>(packed, c);
    self = site_index<DIM>(g, c);
    const uint32_t d = s >> 1;
    uint32_t cd = c[0], st = 1, sh = 0;
#pragma unroll
    for (int k = 1; k < DIM; ++k)
        if (d == (uint32_t)k) {
            cd = c[k];
            st = axis_stride<DIM>(g, k);
            sh = Pack<DIM>::shift(k);
        }
    const uint32_t nc = (s & 1u) ? (cd == 0 ? g.L - 1 : cd - 1) : (cd + 1 == g.L ? 0u : cd + 1);
    j = self + (nc - cd) * st;
    pj = packed + ((nc - cd) << sh);
    owner = (s & 1u) ? j : self;
}

// Warp: one level of speculative growth, members[lo, n) -> new members
// appended.  One lane per (member, direction) pair: a lane loads one
// neighbour, evaluates the one Philox chain its bond draws from and tries
// one claim, so a level costs the warp about one chain instead of D + 1.
// Returns true when the cluster outgrew cap.
template <int DIM, bool kHelper = false>
__device__ __forceinline__ bool win_level(const StepParams &p, uint32_t *members, uint8_t *amask,
                                          uint8_t *omask, uint32_t *hset, uint32_t hslots,
                                          uint32_t cap,
                                          uint32_t lane, uint32_t &lo, uint32_t &n,
                                          uint32_t sig0bit, uint32_t tlo, uint32_t thi) {
    constexpr uint32_t Z = 2 * DIM;          // directions per member
    constexpr uint32_t PER = 32 / Z;         // members per pass (8 in 2D, 5 in 3D)
    const uint32_t hi = n;
    const uint32_t km = lane / Z, s = lane % Z;
    const uint32_t lt = (1u << lane) - 1u;
    bool too_big = false;
    for (uint32_t b = lo; b < hi && !too_big; b += PER) {
        const uint32_t k = b + km;
        const bool act = km < PER && k < hi;
        uint32_t j = 0, pj = 0;
        bool par = false, open = false;
        if (act) {
            uint32_t self, owner;
            neighbour_of<DIM>(p.g, members[k], s, self, j, pj, owner);
            const uint32_t v = grow_read<kHelper>(p.spins + j);
            Philox4 draw;
            philox4x32_10_lanes<1>(&owner, tlo, thi, kTagBond, p.key0, p.key1, &draw);
            const uint32_t d = s >> 1;
            const uint32_t r = d == 0 ? draw.v[0] : d == 1 ? draw.v[1] : draw.v[2];
            par = (uint32_t)(v & 1u) == sig0bit;
            open = (unsigned long long)r < p.thr;
        }
        const bool cand = par && open;
        // the member's alignment and open-bond masks, as its Z lanes read them
        const uint32_t pm = __ballot_sync(kFullMask, par);
        const uint32_t om = __ballot_sync(kFullMask, open);
        if (act && s == 0) {
            amask[k] = (uint8_t)((pm >> (km * Z)) & ((1u << Z) - 1u));
            omask[k] = (uint8_t)((om >> (km * Z)) & ((1u << Z) - 1u));
        }
        bool fresh = false, full = false;
        if (cand) {
            const uint32_t prev = atomicCAS(hset + set_hash(j, hslots), kEmptyKey, j);
            int ins;
            if (prev == kEmptyKey) ins = 1;
            else if (prev == j) ins = 0;
            else ins = set_insert(hset, hslots, j);
            fresh = ins > 0;
            full = ins < 0;
        }
        const uint32_t fm = __ballot_sync(kFullMask, fresh);
        if (fresh) {
            const uint32_t pos = n + __popc(fm & lt);
            if (pos < cap) members[pos] = pj;
            // a member added along y or z expands next level into the row
            // beyond it (and, in 3D, the planes beside it): start those lines
            if (!kHelper && s >= 2) prefetch_two_hop<DIM>(p.g, p.spins, j, s);
        }
        n += __popc(fm);
        if (__any_sync(kFullMask, full) || n > cap) too_big = true;
    }
    __syncwarp();
    lo = hi;
    return too_big;
}

// Warp: sum over the boundary bonds of the grown cluster of (the neighbour is
// parallel ? -1 : +1), i.e. dE_bond / 2 of flipping it (every lane gets it);
// one lane per (member, direction) pair.
template <int DIM>
__device__ __forceinline__ int win_boundary(const StepParams &p, const uint32_t *members,
                                            const uint8_t *amask, uint8_t *bmask,
                                            const uint32_t *hset, uint32_t hslots, uint32_t n,
                                            uint32_t lane) {
    constexpr uint32_t Z = 2 * DIM;
    constexpr uint32_t PER = 32 / Z;
    const uint32_t km = lane / Z, s = lane % Z;
    int dE = 0;
    for (uint32_t b = 0; b < n; b += PER) {
        const uint32_t k = b + km;
        const bool act = km < PER && k < n;
        bool outside = false;
        if (act) {
            uint32_t self, j, pj, owner;
            neighbour_of<DIM>(p.g, members[k], s, self, j, pj, owner);
            const uint32_t home = hset[set_hash(j, hslots)];
            // the neighbour's alignment as the growth read it: the lattice
            // has not changed under it since (a commit that flips a site of
            // the read set restarts the update)
            const bool par = (amask[k] >> s) & 1u;
            // the home slot settles membership unless it holds another site
            outside = !(home == j || (home != kEmptyKey && set_contains(hset, hslots, j)));
            if (outside) dE += par ? -1 : 1;
        }
        const uint32_t bm = __ballot_sync(kFullMask, outside);
        if (act && s == 0) bmask[k] = (uint8_t)((bm >> (km * Z)) & ((1u << Z) - 1u));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(kFullMask, dE, o);
    return dE;
}

// ---- pre-grown updates -------------------------------------------------------
// In a one-lattice launch the clusters after the first (the helpers) grow the
// launch's updates ahead of the main team, in update order, on the lattice as
// they read it while the main team commits, and leave each result in the ring
// (see kRingSlots).  When the main team takes a fresh update it first looks
// there: a result whose read set -- the members, which must still hold the
// seed spin, and each member's neighbours, whose alignment with the seed spin
// must still be what the growth read -- is unchanged on the lattice now is the
// cluster the main team would grow (section 2's cluster depends only on those
// spins and on the counter-based bond draws), with the same levels and
// boundary sum.  The main team never waits for a helper; it grows whatever is
// not there or no longer holds.

__device__ __forceinline__ uint8_t *ring_slot(const StepParams &p, unsigned long long u) {
    return p.ring + (size_t)(u % kRingSlots) * kRingSlotBytes;
}

// The tag of launch update u: the launch's epoch and u + 1, so that a result
// left by an earlier launch (which may have run the same update indices from
// a restored lattice) is never taken.
__device__ __forceinline__ unsigned long long ring_tag(const StepParams &p, unsigned long long u) {
    return ((unsigned long long)p.pg_epoch << 32) | (unsigned long long)(uint32_t)(u + 1);
}

// Warp (main team): takes the pre-grown result of launch update u into the
// window slot (members, masks, meta) if it is there and its read set holds on
// the current lattice.  Returns true if taken (every lane).
template <int DIM>
__device__ __forceinline__ bool take_pregrown(const StepParams &p, unsigned long long u,
                                              uint32_t cap, uint32_t *members, uint8_t *amask,
                                              uint8_t *omask, uint8_t *bmask, uint4 &meta,
                                              uint32_t lane) {
    constexpr uint32_t Z = 2 * DIM;
    constexpr uint32_t PER = 32 / Z;
    const uint8_t *slot = ring_slot(p, u);
    unsigned long long tag = 0;
    if (lane == 0) tag = ld_acquire_u64(reinterpret_cast<const unsigned long long *>(slot));
    tag = __shfl_sync(kFullMask, tag, 0);
    if (tag != ring_tag(p, u)) return false;
    __syncwarp();   // every lane's reads below follow lane 0's acquire
    // the meta word and the first 32 members with their masks in one round
    // trip (a lane past |C| reads bytes it then ignores)
    const uint32_t *rm = reinterpret_cast<const uint32_t *>(slot + kRingMembersOff);
    const uint8_t *ra = slot + kRingMasksOff;
    meta = __ldcg(reinterpret_cast<const uint4 *>(slot + 16));
    const uint32_t mk = __ldcg(rm + lane);
    const uint32_t ak = __ldcg(ra + lane);
    const uint32_t ok = __ldcg(ra + kRingMaxCap + lane);
    const uint32_t bk = __ldcg(ra + 2 * kRingMaxCap + lane);
    const uint32_t n = meta.x;
    if (n == 0 || n > cap) return false;
    if (lane < n) {
        members[lane] = mk;
        amask[lane] = (uint8_t)ak;
        omask[lane] = (uint8_t)ok;
        bmask[lane] = (uint8_t)bk;
    }
    for (uint32_t k = lane + 32; k < n; k += 32) {
        members[k] = __ldcg(rm + k);
        amask[k] = __ldcg(ra + k);
        omask[k] = __ldcg(ra + kRingMaxCap + k);
        bmask[k] = __ldcg(ra + 2 * kRingMaxCap + k);
    }
    __syncwarp();
    // the read set on the current lattice: one lane per (member, direction)
    const uint32_t sig = meta.w;
    const uint32_t km = lane / Z, s = lane % Z;
    bool bad = false;
    for (uint32_t b = 0; b < n; b += PER) {
        const uint32_t k = b + km;
        // the first pass takes the member from the lane that loaded it
        const uint32_t mem = __shfl_sync(kFullMask, mk, km);
        if (km < PER && k < n) {
            uint32_t self, j, pj, owner;
            neighbour_of<DIM>(p.g, b == 0 ? mem : members[k], s, self, j, pj, owner);
            const bool par = (__ldca(p.spins + j) & 1u) == sig;
            if (par != (((uint32_t)amask[k] >> s) & 1u)) bad = true;
            if (s == 0 && (__ldca(p.spins + self) & 1u) != sig) bad = true;
        }
    }
    return !__any_sync(kFullMask, bad);
}

// Helper teams: every warp pre-grows launch updates in order into the ring,
// staying within kRingSlots updates of the main team's commits, until the
// launch's updates are handed out or the main team has finished.  Waits are
// bounded (the wait limit of the launch); a helper that gives up just stops:
// nothing waits for it.
template <int DIM>
__device__ void team_helper(const StepParams &p, TeamShared &sh, const WinCfg &wc) {
    extern __shared__ __align__(16) uint32_t win_dyn[];
    const uint32_t W = min((uint32_t)(blockDim.x >> 5), (uint32_t)kWinMaxWarps);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= W || p.ring == nullptr || wc.slots == 0) return;
    const uint32_t cap = min(wc.cap, kRingMaxCap), hslots = 2 * wc.cap;
    uint32_t *hset = &sh.front[0][0] + warp * hslots;
    // per warp in the dynamic shared memory: members, then the three masks
    const uint32_t stride = cap + (3 * cap + 3) / 4;
    uint32_t *members = win_dyn + warp * stride;
    uint8_t *am = reinterpret_cast<uint8_t *>(members + cap);
    uint8_t *om = am + cap;
    uint8_t *bm = om + cap;
    DevCtl *ctl = p.ctl;
    const uint32_t e = p.pg_epoch & 1u;
    while (true) {
        uint32_t u = 0, go = 1;
        if (lane == 0) {
            if (ld_volatile_u32(&ctl->pg_stop[e])) go = 0;
            else u = atomicAdd(&ctl->pg_next[e], 1u);
            if (go && u >= p.n) go = 0;
            // stay within the ring: slot u mod R is free once the main team
            // has committed update u - R
            const unsigned long long w0 = global_ns();
            while (go && u >= ld_volatile_u32(&ctl->pg_commit[e]) + p.pg_lead) {
                if (ld_volatile_u32(&ctl->pg_stop[e]) || global_ns() - w0 > p.wait_ns) go = 0;
                else __nanosleep(4000);
            }
        }
        go = __shfl_sync(kFullMask, go, 0);
        if (!go) return;
        u = __shfl_sync(kFullMask, u, 0);
        const unsigned long long t = p.t0 + u;
        uint32_t n, lo, levels, sig;
        win_start<DIM, true>(p, seed_site(p, t), members, hset, hslots, lane, n, lo, levels, sig);
        bool big = false;
        while (lo < n && !big) {
            big = win_level<DIM, true>(p, members, am, om, hset, hslots, cap, lane, lo, n, sig,
                                       (uint32_t)t, (uint32_t)(t >> 32));
            ++levels;
        }
        uint8_t *slot = ring_slot(p, u);
        uint4 meta = make_uint4(0u, 0u, 0u, 0u);   // |C| = 0: too big to pre-grow
        if (!big) {
            const int dE = win_boundary<DIM>(p, members, am, bm, hset, hslots, n, lane);
            meta = make_uint4(n, levels, (uint32_t)dE, sig);
            uint32_t *rm = reinterpret_cast<uint32_t *>(slot + kRingMembersOff);
            uint8_t *ra = slot + kRingMasksOff;
            for (uint32_t k = lane; k < n; k += 32) {
                rm[k] = members[k];
                ra[k] = am[k];
                ra[kRingMaxCap + k] = om[k];
                ra[2 * kRingMaxCap + k] = bm[k];
            }
        }
        if (lane == 0) *reinterpret_cast<uint4 *>(slot + 16) = meta;
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            st_release_u64(reinterpret_cast<unsigned long long *>(slot), ring_tag(p, u));
            atomicAdd(&ctl->pg_done[e], 1u);
        }
        __syncwarp();
    }
}

// Warp: a finished update j stamps its flips into the site map,
// list[i] = lowest finished update of the window that flips i.
template <int DIM>
__device__ __forceinline__ void win_stamp(const StepParams &p, const uint32_t *members, uint32_t n,
                                          uint32_t j, uint32_t lane) {
    for (uint32_t k = lane; k < n; k += 32) {
        uint32_t cc[DIM];
        unpack<DIM>(members[k], cc);
        atomicMin(p.list + site_index<DIM>(p.g, cc), j);
    }
}

// Lowest update index below `below` that flips a site of the closed
// neighbourhood of the member `packed` (kNone if none).  The flips of the
// finished updates are stamped into the cluster-list array, which window mode
// uses as a site-indexed map: list[i] = lowest finished update that flips i.
template <int DIM>
__device__ __forceinline__ uint32_t read_conflict(const StepParams &p, uint32_t packed,
                                                  uint32_t below) {
    uint32_t i;
    Neighbours<DIM> nb2;
    neighbours<DIM>(p.g, packed, &i, nb2);
    uint32_t v[2 * DIM + 1];
    v[0] = __ldcg(p.list + i);
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) v[s + 1] = __ldcg(p.list + nb2.idx[s]);
    uint32_t best = kNone;
#pragma unroll
    for (int q = 0; q < 2 * DIM + 1; ++q)
        if (v[q] < below && v[q] < best) best = v[q];
    return best;
}

// A finished update's dependence on an earlier update that flips one of the
// sites it read, for its member `packed` (stamps as in read_conflict, only
// updates below `below` count):
//   rel:   the lowest that flips the member itself or the neighbour across an
//          open boundary bond (rmask).  Those flips change the cluster: section
//          2's cluster holds every site reached through an open bond from a
//          member with the seed spin, and flipping an anti-parallel neighbour
//          across an open bond would add it;
//   any:   the lowest that flips any site read (the member and its boundary
//          neighbours; neighbours that are members check themselves);
//   delta: the change of the update's boundary sum (dE_bond / 2) if every
//          flip of a neighbour across a closed boundary bond (cmask) comes
//          first.  A closed bond never joins its neighbour whatever its spin,
//          so such a flip only turns that bond's term from -1 to +1 or back.
template <int DIM>
__device__ __forceinline__ void check_member(const StepParams &p, uint32_t packed, uint32_t below,
                                             uint32_t rmask, uint32_t cmask, uint32_t amask,
                                             uint32_t &rel, uint32_t &any, int &delta) {
    uint32_t i;
    Neighbours<DIM> nb2;
    neighbours<DIM>(p.g, packed, &i, nb2);
    uint32_t v[2 * DIM + 1];
    v[0] = __ldcg(p.list + i);
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) v[s + 1] = __ldcg(p.list + nb2.idx[s]);
    rel = v[0] < below ? v[0] : kNone;
    any = rel;
    delta = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        if (v[s + 1] >= below) continue;
        if ((rmask >> s) & 1u) rel = min(rel, v[s + 1]);
        if ((cmask >> s) & 1u) {
            any = min(any, v[s + 1]);
            delta += ((amask >> s) & 1u) ? 2 : -2;
        }
    }
    any = min(any, rel);
}

// Block: inclusive scan of three 64-bit sums (blockDim.x <= 512); also
// returns the block totals.
__device__ __forceinline__ void block_scan3(TeamShared &sh, long long &a, long long &b,
                                            long long &c, long long tot[3]) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long ya = __shfl_up_sync(kFullMask, a, o);
        const long long yb = __shfl_up_sync(kFullMask, b, o);
        const long long yc = __shfl_up_sync(kFullMask, c, o);
        if (lane >= (uint32_t)o) {
            a += ya;
            b += yb;
            c += yc;
        }
    }
    if (lane == 31) {
        sh.wsum[0][warp] = a;
        sh.wsum[1][warp] = b;
        sh.wsum[2][warp] = c;
    }
    __syncthreads();
    if (warp == 0) {
        long long x[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) x[q] = lane < nw ? sh.wsum[q][lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const long long y = __shfl_up_sync(kFullMask, x[q], o);
                if (lane >= (uint32_t)o) x[q] += y;
            }
        }
        if (lane < nw) {
#pragma unroll
            for (int q = 0; q < 3; ++q) sh.wsum[q][lane] = x[q];
        }
    }
    __syncthreads();
    if (warp > 0) {
        a += sh.wsum[0][warp - 1];
        b += sh.wsum[1][warp - 1];
        c += sh.wsum[2][warp - 1];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) tot[q] = sh.wsum[q][nw - 1];
    __syncthreads();
}

// Leader CTA: records of the committed updates [c, cut) (relative to u0),
// E_bond and M by a scan of their steps; advances the chain state held by
// thread 0.  Reads the per-slot results of their CTAs remotely.
__device__ void win_records(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                            const WinView &v, uint32_t S, uint32_t cs, unsigned long long u0,
                            uint32_t c, uint32_t cut, long long &E, long long &M,
                            unsigned long long &total_C, uint32_t &last_C,
                            uint32_t &last_levels) {
    if (threadIdx.x == 0) {
        sh.wbase[0] = E;
        sh.wbase[1] = M;
        sh.wbase[2] = (long long)total_C;
    }
    __syncthreads();
    for (uint32_t base = c; base < cut; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        const bool valid = j < cut;
        uint4 m = make_uint4(0, 0, 0, 0);
        if (valid) m = v.lmeta[j - c];
        const uint32_t n = m.x, lev = m.y, sig = m.w;
        const int dE = (int)m.z;
        long long de = valid ? 2LL * dE : 0;
        long long dm = valid ? (sig ? -2LL : 2LL) * (long long)n : 0;
        long long dc = valid ? (long long)n : 0;
        long long tot[3];
        const long long e0 = sh.wbase[0], m0 = sh.wbase[1];
        block_scan3(sh, de, dm, dc, tot);
        if (valid && p.records) {
            wolff_record r;
            r.C = n;
            r.levels = lev;
            r.E_bond = e0 + de;
            r.M = m0 + dm;
            p.records[u0 + j] = r;
        }
        if (j == cut - 1) {
            sh.wlast[0] = n;
            sh.wlast[1] = lev;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            sh.wbase[0] += tot[0];
            sh.wbase[1] += tot[1];
            sh.wbase[2] += tot[2];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        E = sh.wbase[0];
        M = sh.wbase[1];
        total_C = (unsigned long long)sh.wbase[2];
        last_C = sh.wlast[0];
        last_levels = sh.wlast[1];
    }
}

// All CTAs of the team: window mode over updates u0 .. u0 + n_rem - 1 of the
// launch (see the comment at kWinCap).  Returns how many updates it
// committed; the leader's thread 0 holds the advanced chain state.  The
// leader sets wcut = min(n_rem, P), wlimit = kNone and wstop = 0 before the
// phase starts.  The cluster list is the flipped-site map: every slot holds
// kEmptySlot on entry, and again when this returns.
template <int DIM>
__device__ uint32_t team_window(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                                const WinCfg &wc, unsigned long long u0, uint32_t n_rem,
                                unsigned long long launch_t0, long long &E, long long &M,
                                unsigned long long &total_C, uint32_t &last_C,
                                uint32_t &last_levels, unsigned long long &rounds,
                                unsigned long long *win_ns, uint32_t c_start, bool resume,
                                bool &resumable) {
    extern __shared__ __align__(16) uint32_t win_dyn[];
    const uint32_t rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t W = min((uint32_t)(blockDim.x >> 5), (uint32_t)kWinMaxWarps);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = wc.slots, cap = wc.cap, hslots = 2 * cap, K = p.win_levels;
    const uint32_t P = S * cs;
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    uint32_t *hset = &sh.front[0][0] + (warp % kWinMaxWarps) * hslots;
    const WinView v = win_view(win_dyn, S, cap, cs);
    uint32_t c = resume ? c_start : 0;
    if (!resume) {
        for (uint32_t k = threadIdx.x; k < S; k += blockDim.x) v.state[k] = kSlotFree;
        if (threadIdx.x == 0) {
            v.scal[kScNextQ] = 0;
            v.scal[kScSeeded] = 0;
            v.scal[kScRgCount] = 0;
            v.scal[kScRgTake] = 0;
        }
    } else {
        // the window was left for an update too big for it, which has since
        // run the ordinary way: a finished update whose read set (members and
        // their neighbours) changed grows again, the others keep their
        // clusters
        for (uint32_t k = threadIdx.x; k < S; k += blockDim.x) v.cmin[k] = kNone;
        if (warp == 0) win_flatten(v, S, lane);
        __syncthreads();
        const uint32_t total = v.off[S];
        for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
            const uint32_t s = flat_slot(v.off, S, f);
            const uint32_t k = s * cap + (f - v.off[s]);
            const uint32_t sig = v.meta[s].w;
            uint32_t i;
            Neighbours<DIM> nb2;
            neighbours<DIM>(p.g, v.members[k], &i, nb2);
            uint32_t par = 0;
#pragma unroll
            for (int q = 0; q < 2 * DIM; ++q)
                par |= (uint32_t)((__ldcg(p.spins + nb2.idx[q]) & 1u) == sig) << q;
            if ((__ldcg(p.spins + i) & 1u) != sig || par != v.amask[k]) v.cmin[s] = 0;
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < S; k += blockDim.x)
            if (v.state[k] == kSlotDone && v.cmin[k] != kNone) v.state[k] = kSlotRegrow;
        __syncthreads();
        if (warp == 0) win_queue(v, S, c, rank, cs, lane);
    }

    if (wc.helpers && u0 == 0 && !resume) {
        // the launch's first window: give the helpers a moment (bounded) to
        // grow it, instead of growing all of it here while they start.  In
        // 3D the team's other threads meanwhile pull the lattice and the
        // cluster list (the stamps every check and commit reads, 4 bytes a
        // site) into L2, one prefetch per 128-byte line: after the lattice
        // left L2 this cut the 3D L=256 step from 0.547 to 0.505 ms (growth
        // and checks read the six neighbours' stamps line by line at the
        // latency of HBM otherwise).  In 2D the same 81 MB cost the step
        // 13 us (its first window is shorter than the stream), and the
        // lattice alone changed nothing, so 2D does not prefetch.
        if (DIM == 3) {
            const unsigned long long stride = (unsigned long long)cs * blockDim.x * 128ull;
            const unsigned long long first =
                ((unsigned long long)rank * blockDim.x + threadIdx.x) * 128ull;
            for (unsigned long long off = first; off < p.g.N; off += stride)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p.spins + off));
            const uint8_t *lst = reinterpret_cast<const uint8_t *>(p.list);
            for (unsigned long long off = first; off < 4ull * p.g.N; off += stride)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(lst + off));
        }
        if (threadIdx.x == 0) {
            const unsigned int want = min(n_rem, S * cs);
            const unsigned int *done = &p.ctl->pg_done[p.pg_epoch & 1u];
            const unsigned long long w0 = global_ns();
            while (ld_volatile_u32(done) < want && global_ns() - w0 < p.pg_wait_ns)
                __nanosleep(500);
        }
    }
    __syncthreads();
    // this warp's update in progress (registers, kept across rounds)
    bool have = false, restart = false;
    uint32_t g_slot = 0, g_j = 0, g_lo = 0, g_n = 0, g_levels = 0, g_sig = 0;
    const bool timer = win_ns != nullptr && rank == 0 && threadIdx.x == 0;
    unsigned long long tick = timer ? global_ns() : 0;
    uint32_t stall = 0, low_rounds = 0;
    bool first_round = true;
    uint32_t rec_lo = 0, rec_hi = 0;   // committed updates whose records are pending
    resumable = false;
    while (true) {
        const uint32_t lim = min(n_rem, c + P);
        // ---- the finished updates still in the window stamp their flips
        // again (the last commit phase cleared every stamp); updates that
        // finish during this round's growth stamp theirs when they finish
        if (warp == 0) win_flatten(v, S, lane);
        __syncthreads();
        {
            const uint32_t total = v.off[S];
            for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
                const uint32_t s = flat_slot(v.off, S, f);
                uint32_t cc[DIM];
                unpack<DIM>(v.members[s * cap + (f - v.off[s])], cc);
                atomicMin(p.list + site_index<DIM>(p.g, cc), v.j[s]);
            }
        }
        // ---- growth: K levels per warp; fresh updates stop at the first
        // one found too big
        if (threadIdx.x == 0) {
            const uint32_t wl = ld_volatile_u32(&lead->wlimit);
            const uint32_t l2 = min(lim, wl);
            const uint32_t q_end = l2 > rank ? (l2 - rank + cs - 1) / cs : 0;
            v.scal[kScQEnd] = q_end;
            v.scal[kScMin] = kNone;
            const uint32_t seeded = v.scal[kScSeeded];
            v.scal[kScSeedLo] = max(seeded, v.scal[kScNextQ]);
            v.scal[kScSeeded] = max(seeded, q_end);
            if (rank == 0) sh.wcut = lim;
        }
        __syncthreads();
        {
            // the seed sites of the fresh updates this round may hand out
            // (each slot a fresh update will take is free), their lines and
            // the rows their first level reads started towards L1, so that
            // a warp starting one finds them there
            const uint32_t N = p.g.N, L = p.g.L;
            for (uint32_t q = v.scal[kScSeedLo] + threadIdx.x; q < v.scal[kScQEnd];
                 q += blockDim.x) {
                const uint32_t i0 = seed_site(p, p.t0 + u0 + (unsigned long long)(q * cs + rank));
                v.seed[q & (S - 1)] = i0;
                prefetch_l1(p.spins + i0);
                prefetch_l1(p.spins + (i0 + L < N ? i0 + L : i0 + L - N));
                prefetch_l1(p.spins + (i0 >= L ? i0 - L : i0 + N - L));
                if (DIM == 3) {
                    const uint32_t LL = p.g.LL;
                    prefetch_l1(p.spins + (i0 + LL < N ? i0 + LL : i0 + LL - N));
                    prefetch_l1(p.spins + (i0 >= LL ? i0 - LL : i0 + N - LL));
                }
            }
        }
        __syncthreads();
        if (rank == 0 && rec_hi > rec_lo) {
            win_records(p, sh, cl, v, S, cs, u0, rec_lo, rec_hi, E, M, total_C, last_C,
                        last_levels);
            rec_lo = rec_hi = 0;
        }
        if (warp < W) {
            uint32_t steps = 0, pregrown = 0, regrown = 0, grown = 0;
            // with helper teams, an update far beyond the window's head is not
            // needed for this round's commit (rounds commit about 800
            // updates): its warp pauses after K / 3 levels and goes on next
            // round, so that one deep update far out -- typically a pre-grown
            // result a commit invalidated -- does not make the whole round
            // wait.  "Far" is past 3/4 of the window in 2D and past half of it
            // in 3D, the fastest of 1/2, 3/4 and 5/4 on the 10^4-update steps.
            // Without helpers every update is grown here and pausing the far
            // ones only leaves them unfinished when the cut reaches them.
            const uint32_t far_from =
                wc.helpers ? c + (DIM == 2 ? (3u * P) / 4u : P / 2u) : 0xFFFFFFFFu;
            const uint32_t k_far = max(K / 3u, 2u);
            while (steps < K) {
                if (have && g_j >= far_from && steps >= k_far) break;
                bool fresh = false;
                if (!have) {
                    uint32_t took = kNone, tj = 0, fr = 0;
                    if (lane == 0) {
                        // the regrowth queue first (the queue only shrinks
                        // while warps grow, so a plain read may skip it)
                        const uint32_t rg_n = v.scal[kScRgCount];
                        if (ld_volatile_u32(&v.scal[kScRgTake]) < rg_n) {
                            const uint32_t r = atomicAdd(&v.scal[kScRgTake], 1u);
                            if (r < rg_n) {
                                took = v.rg[r];
                                tj = v.j[took];
                            }
                        }
                        if (took == kNone) {
                            // the next fresh update, if below the window's
                            // end (never handed out twice: next_q only grows)
                            const uint32_t q_end = v.scal[kScQEnd];
                            uint32_t q = ld_volatile_u32(&v.scal[kScNextQ]);
                            while (q < q_end) {
                                const uint32_t prev = atomicCAS(&v.scal[kScNextQ], q, q + 1);
                                if (prev == q) {
                                    took = q & (S - 1);
                                    tj = q * cs + rank;
                                    v.j[took] = tj;
                                    fr = 1;
                                    break;
                                }
                                q = prev;
                            }
                        }
                        if (took != kNone) v.state[took] = kSlotGrowing;
                    }
                    took = __shfl_sync(kFullMask, took, 0);
                    tj = __shfl_sync(kFullMask, tj, 0);
                    fresh = __shfl_sync(kFullMask, fr, 0) != 0;
                    if (took == kNone) break;
                    if (!fresh) ++regrown;
                    g_slot = took;
                    g_j = tj;
                    have = true;
                    restart = true;
                }
                const unsigned long long t = p.t0 + u0 + g_j;
                uint32_t *members = v.members + g_slot * cap;
                if (fresh && wc.helpers) {
                    // a fresh update a helper has grown already, if it holds
                    uint4 m;
                    if (take_pregrown<DIM>(p, u0 + g_j, cap, members, v.amask + g_slot * cap,
                                           v.omask + g_slot * cap, v.bmask + g_slot * cap, m,
                                           lane)) {
                        if (lane == 0) {
                            v.meta[g_slot] = m;
                            v.state[g_slot] = kSlotDone;
                        }
                        win_stamp<DIM>(p, members, m.x, g_j, lane);
                        have = false;
                        restart = false;
                        ++steps;
                        ++pregrown;
                        continue;
                    }
                }
                if (restart) {
                    if (fresh) ++grown;
                    win_start<DIM>(p, v.seed[g_slot], members, hset, hslots, lane, g_n, g_lo,
                                   g_levels, g_sig);
                    restart = false;
                }
                const bool big =
                    win_level<DIM>(p, members, v.amask + g_slot * cap, v.omask + g_slot * cap,
                                   hset, hslots, cap, lane,
                                   g_lo, g_n, g_sig, (uint32_t)t, (uint32_t)(t >> 32));
                ++g_levels;
                ++steps;
                if (big) {
                    if (lane == 0) {
                        v.state[g_slot] = kSlotTooBig;
                        atomicMin(&lead->wlimit, g_j);
                    }
                    have = false;
                } else if (g_lo == g_n) {
                    const int dE = win_boundary<DIM>(p, members, v.amask + g_slot * cap,
                                                     v.bmask + g_slot * cap, hset, hslots, g_n,
                                                     lane);
                    if (lane == 0) {
                        v.meta[g_slot] = make_uint4(g_n, g_levels, (uint32_t)dE, g_sig);
                        v.state[g_slot] = kSlotDone;
                    }
                    win_stamp<DIM>(p, members, g_n, g_j, lane);
                    have = false;
                    ++steps;
                }
            }
            if (lane == 0 && steps) atomicAdd(&lead->wlevels, (unsigned long long)steps);
            if (lane == 0 && pregrown)
                atomicAdd(&p.ctl->st_pregrown, (unsigned long long)pregrown);
            if (lane == 0 && regrown)
                atomicAdd(&p.ctl->st_win_regrown, (unsigned long long)regrown);
            if (lane == 0 && grown)
                atomicAdd(&p.ctl->st_win_fresh_grown, (unsigned long long)grown);
        }
        __syncthreads();
        // ---- flatten this CTA's finished updates: off[s] = members before slot s
        if (warp == 0) win_flatten(v, S, lane);
        for (uint32_t k = threadIdx.x; k < S; k += blockDim.x) {
            v.cmin[k] = kNone;
            v.amin[k] = kNone;
            v.dcorr[k] = 0;
        }
        cl.sync();   // every finished update has stamped its flips, every CTA has flattened
        if (timer) {
            const unsigned long long before = win_ns[0];
            win_tick(win_ns[0], tick);
            if (first_round) win_ns[5] += win_ns[0] - before;
        }
        first_round = false;
        if (timer) win_tick(win_ns[1], tick);   // (no separate stamping phase)
        const uint32_t total = v.off[S];
        // ---- conflicts: the lowest earlier update whose flips change each
        // finished update's cluster, and the corrections of its boundary sum
        for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
            const uint32_t s = flat_slot(v.off, S, f);
            const uint32_t k = s * cap + (f - v.off[s]);
            const uint32_t bm = v.bmask[k], om = v.omask[k];
            uint32_t rel, any;
            int delta;
            check_member<DIM>(p, v.members[k], v.j[s], bm & om, bm & ~om, v.amask[k], rel, any,
                              delta);
            if (rel != kNone) atomicMin(&v.cmin[s], rel);
            if (any != kNone) atomicMin(&v.amin[s], any);
            if (delta) atomicAdd(&v.dcorr[s], delta);
        }
        // an update still growing: the lowest update that flips a site it
        // read (it starts again if that one commits)
        uint32_t g_min = kNone;
        if (warp < W && have && !restart) {
            const uint32_t *members = v.members + g_slot * cap;
            for (uint32_t k = lane; k < g_n && k < cap; k += 32)
                g_min = min(g_min, read_conflict<DIM>(p, members[k], kNone));
            g_min = __reduce_min_sync(kFullMask, g_min);
        }
        __syncthreads();
        {
            // the lowest update of this CTA in [c, lim) that cannot commit
            const uint32_t qlo = c > rank ? (c - rank + cs - 1) / cs : 0;
            uint32_t blk = kNone;
            for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
                const uint32_t q = qlo + ((s - qlo) & (S - 1));
                const uint32_t jj = q * cs + rank;
                if (jj < lim) {
                    const bool ok =
                        v.state[s] == kSlotDone && v.j[s] == jj && v.cmin[s] == kNone;
                    if (!ok) blk = min(blk, jj);
                }
            }
            blk = __reduce_min_sync(kFullMask, blk);
            if (lane == 0 && blk != kNone) atomicMin(&v.scal[kScMin], blk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (v.scal[kScMin] != kNone) atomicMin(&lead->wcut, v.scal[kScMin]);
            if (rank == 0 && p.budget_ns)
                sh.wstop = (global_ns() - launch_t0 > p.budget_ns) ? 1u : 0u;
        }
        cl.sync();
        if (timer) win_tick(win_ns[2], tick);
        const uint32_t cut = ld_volatile_u32(&lead->wcut);
        const uint32_t wl = ld_volatile_u32(&lead->wlimit);
        const uint32_t stop = ld_volatile_u32(&lead->wstop);
        if (wc.helpers && rank == 0 && threadIdx.x == 0)   // helpers may reuse slots below it
            *reinterpret_cast<volatile unsigned int *>(&p.ctl->pg_commit[p.pg_epoch & 1u]) =
                (uint32_t)(u0 + cut);
        // ---- commit [c, cut): flip the members (both bits), write records;
        // every stamp is cleared (every read of them ended at the last cluster
        // barrier); the finished updates that stay stamp again next round
        for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
            const uint32_t s = flat_slot(v.off, S, f);
            uint32_t cc[DIM];
            unpack<DIM>(v.members[s * cap + (f - v.off[s])], cc);
            const uint32_t site = site_index<DIM>(p.g, cc);
            p.list[site] = kEmptySlot;
            if (v.j[s] < cut) st_relaxed_u8(p.spins + site, v.meta[s].w ? 0x00u : 0x03u);
        }
        // the leader writes the records of [c, cut) at the start of the next
        // round (or on leaving), off this phase's critical path, from the
        // results pushed here at their offsets from the window start: every
        // update below it commits, so each boundary correction applies
        if (cut > c) {
            rec_lo = c;
            rec_hi = cut;
        }
        uint4 *lead_meta = cl.map_shared_rank(v.lmeta, 0);
        // the committed slots are free; a finished update that read a
        // committed flip grows again
        for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
            if (v.state[s] == kSlotDone) {
                if (v.j[s] < cut) {
                    uint4 m = v.meta[s];
                    m.z = (uint32_t)((int)m.z + v.dcorr[s]);
                    lead_meta[v.j[s] - c] = m;
                    v.state[s] = kSlotFree;
                } else if (v.amin[s] < cut) {
                    v.state[s] = kSlotRegrow;
                }
            }
        }
        // an update still growing that read a committed flip starts again
        if (warp < W && have && !restart && cut > c && g_min < cut) restart = true;
        __syncthreads();
        if (warp == 0) win_queue(v, S, cut, rank, cs, lane);
        ++rounds;
        // the update at the cut finishes within cap / K rounds of its last
        // (re)start, and nothing restarts the lowest uncommitted update
        // twice; a window that stops advancing anyway hands it over and
        // reports the fault
        stall = cut == c ? stall + 1 : 0;
        const bool stuck = stall > kWinMaxStall;
        if (stuck && rank == 0 && threadIdx.x == 0) raise_status(p.ctl, WOLFF_EINVAL, 0xD4u);
        const bool finished = cut >= n_rem;
        const bool blocked = !finished && (cut == wl || stuck);
        const bool stopped = stop != 0 && u0 + cut > 0;
        low_rounds = cut - c < kWinLowYield ? low_rounds + 1 : 0;
        const bool low = !finished && !blocked && low_rounds >= kWinLowRounds;
        cl.sync();   // commits visible, every read of the stamps done
        if (timer) win_tick(win_ns[3], tick);
        c = cut;
        if (finished || blocked || stopped || low) {
            resumable = blocked && !stuck && !stopped;
            if (rank == 0 && threadIdx.x == 0) sh.wlowy = low ? 1u : 0u;
            break;
        }
    }
    if (resumable) {
        // the update at the cut runs the ordinary way; the window keeps its
        // finished updates and regrows the rest when it resumes
        if (warp < W && have && lane == 0) v.state[g_slot] = kSlotRegrow;
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < S; k += blockDim.x)
            if (v.state[k] == kSlotTooBig) v.state[k] = v.j[k] == c ? kSlotFree : kSlotRegrow;
    }
    if (rank == 0 && rec_hi > rec_lo)
        win_records(p, sh, cl, v, S, cs, u0, rec_lo, rec_hi, E, M, total_C, last_C, last_levels);
    // the cluster list is empty (the last commit phase cleared every stamp);
    // order that before whatever uses it next
    cl.sync();
    if (timer) win_ns[4] += sh.wlevels;
    return c;
}

// Leader: announce a team phase, then start it with the cluster barrier.
__device__ __forceinline__ void announce(TeamShared &sh, cg::cluster_group &cl, unsigned int kind,
                                         uint32_t lo, uint32_t hi, uint32_t level,
                                         uint32_t sig0bit, unsigned long long t) {
    if (threadIdx.x == 0) {
        sh.cmd[0] = kind;
        sh.cmd[1] = lo;
        sh.cmd[2] = hi;
        sh.cmd[3] = level;
        sh.cmd[4] = sig0bit;
        sh.cmd[5] = (uint32_t)t;
        sh.cmd[6] = (uint32_t)(t >> 32);
        sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
    }
    cl.sync();
}

template <int DIM>
__device__ void team_leader(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                            const WinCfg &wc) {
    DevCtl *ctl = p.ctl;
    const bool t0 = threadIdx.x == 0;
    const bool has_team = cl.num_blocks() > 1;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long E = 0, M = 0;
    unsigned long long total_C = 0;
    uint32_t last_C = 0, last_levels = 0;
    unsigned long long st_local = 0, st_team = 0, ns_local = 0, ns_team = 0, ns_finish = 0;
    unsigned long long handoffs = 0, team_fin = 0;
    if (t0) {
        ctl->st_start_ns = global_ns();
        E = ctl->E;
        M = ctl->M;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
        sh.dE = 0;
    }
    // window policy (thread 0 decides, the CTA follows): windows run while the
    // recent clusters are small; a cluster too big for one pauses them
    unsigned int cooldown = 0, fail_streak = 0, skip_next = 0;
    unsigned long long window_updates = 0, window_rounds = 0;
    // growth, map, check, commit, growth levels, first round's growth
    unsigned long long win_ns[6] = {0, 0, 0, 0, 0, 0};
    // an open window (left for an update too big for it) resumes at
    // update win_u0 + win_next
    bool win_open = false;
    unsigned long long win_u0 = 0;
    uint32_t win_nrem = 0, win_next = 0;
    unsigned long long life_rounds = 0, life_done = 0;   // windows' rounds and commits since the last back-off
    const unsigned long long launch_t0 = global_ns();
    const uint32_t pg = p.pg_epoch & 1u;
    if (wc.helpers && t0) {
        // the next launch's helper words start from zero (it cannot start
        // before this one has ended, helpers included)
        ctl->pg_next[pg ^ 1u] = 0;
        ctl->pg_stop[pg ^ 1u] = 0;
        ctl->pg_commit[pg ^ 1u] = 0;
        ctl->pg_done[pg ^ 1u] = 0;
    }
    unsigned long long u = 0;
    for (; u < p.n; ++u) {
        if (wc.helpers && t0)
            *reinterpret_cast<volatile unsigned int *>(&ctl->pg_commit[pg]) = (uint32_t)u;
        if (p.budget_ns && u > 0) {   // a time-budgeted job stops at an update boundary
            if (t0) sh.budget_stop = (global_ns() - launch_t0 > p.budget_ns) ? 1u : 0u;
            __syncthreads();
            if (sh.budget_stop) break;
        }
        if (p.win_levels && wc.slots && p.n - u >= 2) {
            // a window stopped by an update too big for it leaves that update
            // to the ordinary path directly, then resumes with what it holds
            const bool resume = win_open && u == win_u0 + win_next;
            if (t0) sh.wflag = (resume || (cooldown == 0 && !skip_next)) ? 1u : 0u;
            __syncthreads();
            if (sh.wflag) {
                const unsigned long long u0w = resume ? win_u0 : u;
                const uint32_t n_rem =
                    resume ? win_nrem : (uint32_t)min(p.n - u, 0x7FFFFFFFull);
                const uint32_t c_start = resume ? win_next : 0;
                if (t0) {
                    sh.wlimit = kNone;
                    sh.wstop = 0;
                    sh.wlevels = 0;
                    sh.wlowy = 0;
                }
                if (has_team)
                    announce(sh, cl, kTeamWindow, (uint32_t)u0w, (uint32_t)(u0w >> 32), n_rem,
                             resume ? 1u : 0u, c_start);
                else
                    __syncthreads();
                bool resumable = false;
                const unsigned long long rounds0 = window_rounds;
                const uint32_t c =
                    team_window<DIM>(p, sh, cl, wc, u0w, n_rem, launch_t0, E, M, total_C, last_C,
                                     last_levels, window_rounds, win_ns, c_start, resume,
                                     resumable);
                const uint32_t done = c - c_start;
                life_rounds += window_rounds - rounds0;
                life_done += done;
                const bool low_life = life_rounds >= kWinLowRounds &&
                                      life_done < (unsigned long long)kWinLowYield * life_rounds;
                if (low_life) {
                    life_rounds = life_done = 0;
                } else if (life_rounds >= 64) {   // recent windows weigh most
                    life_rounds >>= 1;
                    life_done >>= 1;
                }
                if (t0 && low_life) sh.wlowy = 1u;
                __syncthreads();
                // a resumed window that commits nothing is closed, and so is
                // one that commits too little per round
                win_open = resumable && !(resume && done == 0) && !sh.wlowy;
                win_u0 = u0w;
                win_nrem = n_rem;
                win_next = c + 1;
                if (t0) {
                    window_updates += done;
                    if (done > 0 && c < n_rem && !sh.wstop) skip_next = 1;
                    // back off only while fresh windows keep failing at their
                    // first update (the large-cluster regime): 0, 1, 3, ..., 63;
                    // a window left for committing too little per round backs
                    // off the longest way at once
                    if (sh.wlowy) {
                        fail_streak = 7u;
                        cooldown = 63u;
                        skip_next = 0;
                    } else if (done == 0 && !resume) {
                        fail_streak = min(fail_streak + 1u, 7u);
                        cooldown = (1u << (fail_streak - 1u)) - 1u;
                    } else if (done > 0) {
                        fail_streak = 0;
                    }
                }
                if (done > 0) {
                    u = u0w + c - 1;
                    continue;
                }
            } else if (t0) {
                if (skip_next) skip_next = 0;
                else --cooldown;
            }
        }
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        unsigned long long clk = 0;
        if (t0) {
            const uint32_t i0 = seed_site(p, t);
            unsigned int *w = reinterpret_cast<unsigned int *>(p.spins) + (i0 >> 2);
            const unsigned int sh0 = (i0 & 3u) * 8u;
            const uint32_t s0 = (atomicXor(w, 1u << sh0) >> sh0) & 1u;
            const uint32_t p0 = pack_index<DIM>(p.g, i0);
            p.list[0] = p0;
            sh.list[0] = p0;
            sh.front[0][0] = p0;
            sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
            sh.sig0bit = s0;
            clk = global_ns();
        }
        __syncthreads();
        const uint32_t sig0bit = sh.sig0bit;
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_team = false;
        while (f > 0) {
            if (has_team && f > p.t_up) {
                went_team = true;
                unsigned long long g0 = 0;
                if (t0) {
                    g0 = global_ns();
                    ns_local += g0 - clk;
                    ++handoffs;
                }
                announce(sh, cl, kTeamLevels, C - f, C, level, sig0bit, t);
                uint32_t lo = C - f, hi = C, lv0 = level;
                bool finished = false;
                team_levels<DIM>(p, sh, cl, lo, hi, level, sig0bit, tlo, thi, &finished);
                C = hi;
                f = finished ? 0u : hi - lo;
                for (uint32_t k = threadIdx.x; k < f && k < kLocalFrontierCap; k += blockDim.x)
                    sh.front[cur][k] = __ldcg(p.list + lo + k);
                if (t0) {
                    sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                    st_team += level - lv0;
                    clk = global_ns();
                    ns_team += clk - g0;
                }
                __syncthreads();
                continue;
            }
            // one level on the leader alone; a front larger than the shared
            // buffer is read from the cluster list, which this CTA wrote
            const uint32_t nxt = cur ^ 1u;
            const uint32_t fbase = C - f;
            unsigned int *cnt = &sh.cnt[level % 3];
            if (t0) sh.cnt[(level + 1) % 3] = 0;
            for (uint32_t b = warp * 32u; b < f; b += nwarps * 32u) {
                const uint32_t k = b + lane;
                Neighbours<DIM> nb;
                uint32_t won = 0;
                if (k < f) {
                    const uint32_t packed =
                        k < kLocalFrontierCap ? sh.front[cur][k] : __ldcg(p.list + fbase + k);
                    won = expand_site<DIM>(p, packed, sig0bit, tlo, thi, nb);
                }
                uint32_t pos = warp_reserve(cnt, __popc(won));
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (won & (1u << s)) {
                        const uint32_t gpos = C + pos;
                        if (gpos < p.g.N) p.list[gpos] = nb.packed[s];
                        else raise_status(ctl, WOLFF_EINVAL, 0xD3u);
                        if (gpos < kLocalListCap) sh.list[gpos] = nb.packed[s];
                        if (pos < kLocalFrontierCap) sh.front[nxt][pos] = nb.packed[s];
                        ++pos;
                    }
                }
            }
            __syncthreads();
            const uint32_t added = *cnt;
            ++level;
            if (t0) ++st_local;
            C += added;
            f = added;
            cur = nxt;
        }
        long long dE = 0;
        unsigned long long f0 = 0;
        if (t0) {
            f0 = global_ns();
            ns_local += f0 - clk;
        }
        if (went_team || (has_team && C > p.t_up * 4u && C > kLocalListCap)) {
            if (t0) ++team_fin;
            announce(sh, cl, kTeamFinish, 0, C, level, sig0bit, t);
            dE = team_finish<DIM>(p, sh, cl, C, sig0bit);
        } else {
            // the leader closes the cluster alone
            const bool in_shared = C <= kLocalListCap;
            long long acc = 0;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t i;
                acc += boundary_term<DIM>(p, in_shared ? sh.list[k] : __ldcg(p.list + k), sig0bit,
                                          &i);
            }
            dE = block_sum(acc);
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(in_shared ? sh.list[k] : __ldcg(p.list + k), c);
                unmark_site(p.spins, site_index<DIM>(p.g, c), sig0bit);
                p.list[k] = kEmptySlot;
            }
        }
        if (t0) {
            E += 2 * dE;
            M += (sig0bit ? -2LL : 2LL) * (long long)C;
            total_C += C;
            last_C = C;
            last_levels = level;
            if (p.records) {
                wolff_record r;
                r.C = C;
                r.levels = level;
                r.E_bond = E;
                r.M = M;
                p.records[u] = r;
            }
            ns_finish += global_ns() - f0;
        }
        __syncthreads();
    }
    if (t0) {
        ctl->E = E;
        ctl->M = M;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + u;
        ctl->st_updates += u;
        ctl->st_levels_local += st_local;
        ctl->st_levels_grid += st_team;
        ctl->st_ns_local += ns_local;
        ctl->st_ns_grid += ns_team;
        ctl->st_ns_finish += ns_finish;
        ctl->st_handoffs += handoffs;
        ctl->st_grid_finishes += team_fin;
        ctl->st_burst_updates += window_updates;
        ctl->st_bursts += window_rounds;
        for (int k = 0; k < 4; ++k) ctl->st_ns_win[k] += win_ns[k];
        ctl->st_win_levels += win_ns[4];
        ctl->st_ns_win_first += win_ns[5];
        ctl->st_end_ns = global_ns();
        if (wc.helpers) *reinterpret_cast<volatile unsigned int *>(&ctl->pg_stop[pg]) = 1u;
    }
    if (has_team) {
        announce(sh, cl, kTeamExit, 0, 0, 0, 0, 0);
        cl.sync();   // no CTA of the team exits while another may still read its shared memory
    }
}

template <int DIM>
__global__ void __launch_bounds__(512, 1) k_team(StepParams single, const StepParams *table,
                                                 WinCfg wc) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ TeamShared sh;
    const unsigned int job = blockIdx.x / cl.num_blocks();
    if (wc.helpers && job > 0) {   // a one-lattice launch's pre-growing helper team
        team_helper<DIM>(single, sh, wc);
        return;
    }
    const StepParams p = table ? table[job] : single;
    if (cl.block_rank() != 0) {
        team_worker<DIM>(p, sh, cl, wc);
        return;
    }
    team_leader<DIM>(p, sh, cl, wc);
}

// Kernel attributes already set, per device and dimension.
constexpr int kAttrDevices = 64;
std::atomic<bool> g_nonportable_set[kAttrDevices][2];
std::atomic<size_t> g_dyn_smem_set[kAttrDevices][2];

}  // namespace

const void *team_kernel(int dim) {
    return dim == 2 ? reinterpret_cast<const void *>(&k_team<2>)
                    : reinterpret_cast<const void *>(&k_team<3>);
}

cudaError_t ensure_team_dyn_smem(int dim, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrDevices) {
        cudaGetLastError();
        return cudaFuncSetAttribute(team_kernel(dim), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes);
    }
    // the attribute is an upper bound: it only ever grows to the largest
    // request, so a value recorded here is never above the real one
    std::atomic<size_t> &cur = g_dyn_smem_set[dev][dim == 2 ? 0 : 1];
    size_t seen = cur.load();
    if (bytes <= seen) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(team_kernel(dim),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    while (seen < bytes && !cur.compare_exchange_weak(seen, bytes)) {
    }
    return cudaSuccess;
}

// Members per speculative update: 64 with 16 warps per CTA in 2D, 128 in 3D
// (where the random-start clusters reach ~90) and whenever a CTA has 8 warps
// or fewer.  The per-warp hash sets (2 cap entries each) fill at most half of
// the TeamShared raw area.
uint32_t window_cap(int dim, int threads) {
    const uint32_t W = min((uint32_t)threads / 32u, (uint32_t)kWinMaxWarps);
    return (W <= 8 || dim == 3) ? 2 * kWinCap : kWinCap;
}

size_t window_smem_bytes(int dim, int threads, int window_slots, int cluster_size) {
    if (window_slots <= 0) return 0;
    const size_t cap = window_cap(dim, threads);
    const size_t S = (size_t)window_slots;
    return (S * cap + 12 * S + 1 + kWinScalars + 4 * S * (size_t)cluster_size) * sizeof(uint32_t) +
           3 * S * cap;
}

cudaError_t launch_team(int dim, const StepParams &single, const StepParams *d_table, int njobs,
                        int cluster_size, int threads, int window_slots, cudaStream_t s,
                        int helpers) {
    if (njobs <= 0) return cudaSuccess;
    if (helpers < 0 || (helpers > 0 && (d_table != nullptr || njobs != 1 || window_slots == 0 ||
                                        single.ring == nullptr)))
        return cudaErrorInvalidValue;
    if (window_slots < 0 || (window_slots & (window_slots - 1)) != 0 || window_slots > 1024)
        return cudaErrorInvalidValue;
    const void *fn = team_kernel(dim);
    // kernel attributes are set once per device and value (a driver call per
    // launch otherwise)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrDevices) {
        cudaGetLastError();
        dev = -1;
    }
    const int di = dim == 2 ? 0 : 1;
    if (cluster_size > 8 && (dev < 0 || !g_nonportable_set[dev][di].load())) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        if (dev >= 0) g_nonportable_set[dev][di].store(true);
    }
    WinCfg wc;
    wc.slots = (uint32_t)window_slots;
    wc.cap = window_cap(dim, threads);
    wc.helpers = (uint32_t)helpers;
    const size_t dyn = window_smem_bytes(dim, threads, window_slots, cluster_size);
    if (dyn > 0) {
        cudaError_t e = ensure_team_dyn_smem(dim, dyn);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((njobs + helpers) * cluster_size));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<StepParams *>(&single), const_cast<StepParams **>(&d_table), &wc};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int team_max_active_clusters(int dim, int cluster_size, int threads, int window_slots) {
    const void *fn = team_kernel(dim);
    const size_t dyn = window_smem_bytes(dim, threads, window_slots, cluster_size);
    if (cluster_size > 8 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dyn > 0 && ensure_team_dyn_smem(dim, dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster_size);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace wolff
