// wolff_tiny.cu -- the single-cluster update of section 2 for lattices of at
// most kTinyMaxSites sites, one CTA per lattice, the lattice held in shared
// memory as bit planes for the whole launch.
//
// The paper finds the CPU faster than the GPU on small lattices (section 5,
// Tables 1-2): every level of the wave front pays a grid-wide
// synchronisation however few spins it holds.  Here a level is a handful of
// word operations inside one SM.  Each lattice row (fixed y, z) is a string
// of L bits split into W = ceil(L/32) 32-bit words; a breadth-first level
// computes the next wave front of every word at once,
//   new = (fwd_x(F & OX) | bwd_x(F) & OX | F[row-1] & OY[row-1] | F[row+1] & OY
//          [| the same along z]) & A & ~V,
// where F is the wave front, V the cluster so far, A the sites parallel to
// the seed spin, and OX/OY/OZ the bonds (i, d) whose draw r_d(i) < thr
// (bit x of a word belongs to the bond's owner, section 2's undirected bond
// id: the forward bond of site x).  The component of the seed in the graph
// of open bonds between sites parallel to the seed spin -- the cluster -- and
// the number of breadth-first generations are those of the serial update,
// whatever the traversal, so the records equal the other schedules' bit for
// bit.  E_bond and M are recounted from their definitions after every flip
// with population counts (D N - 2 x anti-parallel bonds, 2 x up spins - N).
//
// Two regimes, by the number of words NW = (N / L) W:
//   - NW <= 64 (2D L <= 32, 3D L <= 8, where a row is one word) with 64 or
//     more threads: warp 0 alone runs the update with its rows in registers
//     (one or two per lane), neighbour rows fetched by shuffles, a level
//     ended by one vote; the other warps draw the next update's bond bits
//     and seed meanwhile (a draw depends only on (seed, t, bond), never on
//     the spins), so the Philox work is hidden;
//   - otherwise every thread owns one or two words; the update's draws come
//     first, then levels separated by __syncthreads_or, which also tells
//     whether the wave front is empty.
//
// Shared memory (32-bit words): S[NW] spins (1 = +1; in warp mode only at
// the launch's start and end, warp 0 holds them meanwhile) | B[2][DIM][NW]
// open bonds by update parity and axis | F[2][NW] wave front, ping-pong (the
// all-thread regime) | 8 words of sums.  The lattice is read from the
// workspace at the start of a launch and written back (bit 0 = bit 1 = spin)
// at its end.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "wolff_device.cuh"
#include "wolff_internal.h"
#include "wolff_tiny.h"

namespace wolff {
namespace {

struct TinyGeo {
    uint32_t L, N, W, NW;
    uint32_t hb;         // bit of site x = L-1 in its word
    uint32_t lastmask;   // valid bits of a row's last word
    __host__ __device__ explicit TinyGeo(uint32_t L_, uint32_t N_) : L(L_), N(N_) {
        W = (L + 31u) / 32u;
        NW = (N / L) * W;
        hb = (L - 1u) & 31u;
        lastmask = hb == 31u ? 0xffffffffu : (1u << (hb + 1u)) - 1u;
    }
};

// smem offsets (32-bit words)
__host__ __device__ inline uint32_t off_bonds(const TinyGeo &g) { return g.NW; }
template <int DIM>
__host__ __device__ inline uint32_t off_front(const TinyGeo &g) { return g.NW * (1u + 2u * DIM); }
template <int DIM>
__host__ __device__ inline uint32_t off_sums(const TinyGeo &g) { return g.NW * (3u + 2u * DIM); }
template <int DIM>
__host__ __device__ inline uint32_t tiny_words(const TinyGeo &g) { return off_sums<DIM>(g) + 8u; }

// One word's fixed neighbourhood: its row-neighbour words along x (previous
// and next word of the row, cyclically) and the same word of the rows before
// and after along y (and z).
template <int DIM>
struct WordNb {
    uint32_t k, w;
    uint32_t kxp, kxn;     // words holding sites 32w - 1 and 32w + 32 (cyclic in the row)
    uint32_t cbit;         // bit of site 32w - 1 in word kxp (31, or hb when w = 0)
    uint32_t qpos;         // bit that receives site 32w + 32 (31, or hb when w = W-1)
    uint32_t ym, yp, zm, zp;
    uint32_t vm;           // valid bits
};

template <int DIM>
__device__ __forceinline__ WordNb<DIM> word_nb(const TinyGeo &g, uint32_t k) {
    WordNb<DIM> n;
    n.k = k;
    const uint32_t r = k / g.W, w = k - r * g.W;
    n.w = w;
    n.kxp = w == 0u ? k + (g.W - 1u) : k - 1u;
    n.kxn = w == g.W - 1u ? k - (g.W - 1u) : k + 1u;
    n.cbit = w == 0u ? g.hb : 31u;
    n.qpos = w == g.W - 1u ? g.hb : 31u;
    n.vm = w == g.W - 1u ? g.lastmask : 0xffffffffu;
    const uint32_t y = DIM == 2 ? r : r % g.L;
    const uint32_t rowW = g.W;                 // words between rows y and y + 1
    n.ym = y == 0u ? k + (g.L - 1u) * rowW : k - rowW;
    n.yp = y == g.L - 1u ? k - (g.L - 1u) * rowW : k + rowW;
    n.zm = n.zp = k;
    if (DIM == 3) {
        const uint32_t z = r / g.L, slab = g.L * g.W;
        n.zm = z == 0u ? k + (g.L - 1u) * slab : k - slab;
        n.zp = z == g.L - 1u ? k - (g.L - 1u) * slab : k + slab;
    }
    return n;
}

// The bond bits of the update with counter t for every word handled by this
// warp (words wi, wi + nw, ...): lane x of a word draws the site 32w + x,
// and a ballot per axis packs the bits (bit set = r_d < thr).  Four words
// per pass run their Philox chains interleaved.
template <int DIM>
__device__ __forceinline__ void draw_words(const StepParams &p, const TinyGeo &g,
                                           unsigned long long t, uint32_t *B, uint32_t wi,
                                           uint32_t nw) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t k0 = wi; k0 < g.NW; k0 += 4u * nw) {
        uint32_t site[4];
        bool valid[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t k = k0 + (uint32_t)q * nw;
            const uint32_t r = k / g.W, w = k - r * g.W;
            const uint32_t x = 32u * w + lane;
            valid[q] = k < g.NW && x < g.L;
            site[q] = valid[q] ? x + g.L * r : 0u;
        }
        Philox4 d[4];
        philox4x32_10_lanes<4>(site, (uint32_t)t, (uint32_t)(t >> 32), kTagBond, p.key0, p.key1,
                               d);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t k = k0 + (uint32_t)q * nw;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const uint32_t bits = __ballot_sync(
                    kFullMask, valid[q] && (unsigned long long)d[q].v[a] < p.thr);
                if (lane == (uint32_t)a && k < g.NW) B[a * g.NW + k] = bits;
            }
        }
    }
}

// The same for rows of at most 16 sites (one word each): R = 2^lr rows share
// a warp's draw, 2^ls = 32 / R lanes a row (the power of two at or above L),
// so short rows leave no lanes idle; row j's bits are bits [j 2^ls,
// j 2^ls + L) of the ballot.  The warp handles units of R rows (wi, wi + nw,
// ...), four units per pass.
template <int DIM>
__device__ __forceinline__ void draw_short_rows(const StepParams &p, const TinyGeo &g,
                                                unsigned long long t, uint32_t *B, uint32_t wi,
                                                uint32_t nw) {
    uint32_t ls = 4u;   // the power of two at or above L (L <= 16)
    while (ls > 0u && (1u << (ls - 1u)) >= g.L) --ls;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lr = 5u - ls;
    const uint32_t sub = lane >> ls, x = lane & ((1u << ls) - 1u);
    const uint32_t rowmask = (1u << g.L) - 1u;
    const uint32_t units = (g.NW + (1u << lr) - 1u) >> lr;
    for (uint32_t u0 = wi; u0 < units; u0 += 4u * nw) {
        uint32_t site[4];
        bool valid[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t r = ((u0 + (uint32_t)q * nw) << lr) + sub;   // the row is the word
            valid[q] = r < g.NW && x < g.L;
            site[q] = valid[q] ? x + g.L * r : 0u;
        }
        Philox4 d[4];
        philox4x32_10_lanes<4>(site, (uint32_t)t, (uint32_t)(t >> 32), kTagBond, p.key0, p.key1,
                               d);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // lane j < R writes row j of the unit
            const uint32_t k = ((u0 + (uint32_t)q * nw) << lr) + lane;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const uint32_t bits = __ballot_sync(
                    kFullMask, valid[q] && (unsigned long long)d[q].v[a] < p.thr);
                if ((lane >> lr) == 0u && k < g.NW) B[a * g.NW + k] = (bits >> (lane << ls)) & rowmask;
            }
        }
    }
}

// SHORT: a kernel instantiation for lattices whose rows are at most 16
// sites (one word each); the others draw word by word.  Each instantiation
// carries one of the two, so neither's registers weigh on the other's loops.
template <int DIM, bool SHORT>
__device__ __forceinline__ void draw_bonds(const StepParams &p, const TinyGeo &g,
                                           unsigned long long t, uint32_t *B, uint32_t wi,
                                           uint32_t nw) {
    if (SHORT)
        draw_short_rows<DIM>(p, g, t, B, wi, nw);
    else
        draw_words<DIM>(p, g, t, B, wi, nw);
}

__device__ __forceinline__ uint32_t seed_of(const StepParams &p, unsigned long long t,
                                            uint32_t N) {
    const Philox4 r = philox4x32_10(0u, (uint32_t)t, (uint32_t)(t >> 32), kTagSeed, p.key0,
                                    p.key1);
    return (uint32_t)(((unsigned long long)r.v[0] * N) >> 32);
}

// Per-word state of the running update.
struct WordState {
    uint32_t A, V, F;
    uint32_t ox, oxc, oy, oym, oz, ozm;
};

// The next wave front of one word from the current one (Fc: the ping-pong
// half being read).
template <int DIM>
__device__ __forceinline__ uint32_t grow_word(const WordNb<DIM> &n, const WordState &s,
                                              const uint32_t *Fc) {
    // +x: site x-1 -> x across the bond owned by x-1
    const uint32_t cin = (Fc[n.kxp] >> n.cbit) & s.oxc & 1u;
    const uint32_t P = ((s.F & s.ox) << 1) | cin;
    // -x: site x+1 -> x across the bond owned by x
    const uint32_t Q = ((s.F >> 1) | ((Fc[n.kxn] & 1u) << n.qpos)) & s.ox;
    // +y / -y (and z): the bond of the lower row's site, or the word's own
    uint32_t G = P | Q | (Fc[n.ym] & s.oym) | (Fc[n.yp] & s.oy);
    if (DIM == 3) G |= (Fc[n.zm] & s.ozm) | (Fc[n.zp] & s.oz);
    return G & s.A & ~s.V & n.vm;
}

// Loads a word's bond bits for the running update and starts its cluster:
// A = sites parallel to the seed spin, V = F = the seed bit if it is here.
template <int DIM>
__device__ __forceinline__ void start_word(const WordNb<DIM> &n, const TinyGeo &g,
                                           const uint32_t *S, const uint32_t *B, uint32_t sig0bit,
                                           uint32_t seedk, uint32_t seedbit, WordState &s) {
    const uint32_t spins = S[n.k];
    s.A = (sig0bit ? spins : ~spins) & n.vm;
    s.V = s.F = n.k == seedk ? seedbit : 0u;
    s.ox = B[n.k];
    s.oxc = B[n.kxp] >> n.cbit;
    s.oy = B[g.NW + n.k];
    s.oym = B[g.NW + n.ym];
    s.oz = s.ozm = 0u;
    if (DIM == 3) {
        s.oz = B[2u * g.NW + n.k];
        s.ozm = B[2u * g.NW + n.zm];
    }
}

// Anti-parallel forward bonds and up spins of one word (after the flip).
template <int DIM>
__device__ __forceinline__ void count_word(const WordNb<DIM> &n, const uint32_t *S,
                                           uint32_t &anti, uint32_t &up) {
    const uint32_t s = S[n.k];
    const uint32_t sn = (s >> 1) | ((S[n.kxn] & 1u) << n.qpos);   // site x+1's spin at bit x
    uint32_t a = __popc((s ^ sn) & n.vm) + __popc((s ^ S[n.yp]) & n.vm);
    if (DIM == 3) a += __popc((s ^ S[n.zp]) & n.vm);
    anti += a;
    up += __popc(s & n.vm);
}

// ---- warp mode: warp 0 alone, one word per row (W = 1 whenever a lattice
// has at most 64 words), its words' state in registers; a neighbour row
// comes from the lane holding it by a shuffle, so a level costs no shared
// memory traffic and no barrier beyond the vote that ends it.

// Row k of a lattice whose rows are spread over the lanes as v[k / 32] of
// lane k % 32 (every lane calls it; each asks for its own k).
template <int J>
__device__ __forceinline__ uint32_t row_of(const uint32_t (&v)[J], uint32_t k) {
    uint32_t out = __shfl_sync(kFullMask, v[0], k & 31u);
    if (J == 2) {
        const uint32_t hi = __shfl_sync(kFullMask, v[J - 1], k & 31u);
        if (k >> 5) out = hi;
    }
    return out;
}

// One update on warp 0: grows the cluster of seed site i0 level by level,
// flips it in Sr (the warp's rows, kept in registers between updates) and
// returns |C|, the anti-parallel bonds and the up spins after the flip (warp
// sums) and the number of generations.
template <int DIM, int J>
__device__ __forceinline__ void warp_update(const TinyGeo &g, const WordNb<DIM> (&nb)[J],
                                            const bool (&own)[J], uint32_t (&Sr)[J],
                                            const uint32_t *B, uint32_t i0, uint32_t &C,
                                            uint32_t &anti, uint32_t &up, uint32_t &level) {
    const uint32_t x0 = i0 % g.L, r0 = i0 / g.L;
    const uint32_t sig0bit = (row_of<J>(Sr, r0) >> x0) & 1u;
    const uint32_t hb = g.hb;
    uint32_t A[J], V[J], F[J], ox[J], oy[J], oym[J], oz[J], ozm[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t k = nb[j].k;
        A[j] = own[j] ? (sig0bit ? Sr[j] : ~Sr[j]) & nb[j].vm : 0u;
        V[j] = F[j] = (own[j] && k == r0) ? 1u << x0 : 0u;
        ox[j] = B[k];
        oy[j] = B[g.NW + k];
        oym[j] = B[g.NW + nb[j].ym];
        oz[j] = ozm[j] = 0u;
        if (DIM == 3) {
            oz[j] = B[2u * g.NW + k];
            ozm[j] = B[2u * g.NW + nb[j].zm];
        }
    }
    level = 0;
    for (;;) {
        uint32_t nf[J];
        uint32_t any = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const uint32_t gx = F[j] & ox[j];
            // +x across the bond of site x-1, -x across the site's own (a
            // rotation within the row's L bits)
            uint32_t G = ((gx << 1) | ((gx >> hb) & 1u)) |
                         (((F[j] >> 1) | ((F[j] & 1u) << hb)) & ox[j]);
            G |= (row_of<J>(F, nb[j].ym) & oym[j]) | (row_of<J>(F, nb[j].yp) & oy[j]);
            if (DIM == 3)
                G |= (row_of<J>(F, nb[j].zm) & ozm[j]) | (row_of<J>(F, nb[j].zp) & oz[j]);
            nf[j] = G & A[j] & ~V[j];
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            V[j] |= nf[j];
            F[j] = nf[j];
            any |= nf[j];
        }
        ++level;
        if (!__any_sync(kFullMask, any != 0u)) break;
    }
    uint32_t c = 0, a = 0, u = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        Sr[j] ^= V[j];
        c += __popc(V[j]);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t sp = Sr[j];
        const uint32_t sn = (sp >> 1) | ((sp & 1u) << hb);   // site x+1's spin at bit x
        uint32_t aa = __popc((sp ^ sn) & nb[j].vm) +
                      __popc((sp ^ row_of<J>(Sr, nb[j].yp)) & nb[j].vm);
        if (DIM == 3) aa += __popc((sp ^ row_of<J>(Sr, nb[j].zp)) & nb[j].vm);
        if (own[j]) {
            a += aa;
            u += __popc(sp & nb[j].vm);
        }
    }
    C = __reduce_add_sync(kFullMask, c);
    anti = __reduce_add_sync(kFullMask, a);
    up = __reduce_add_sync(kFullMask, u);
}

// CTAs are capped at 768 threads in 2D (80 registers a thread) and 512 in 3D
// (128): a 2D lattice has at most 1086 words and a 3D one 1024, two per
// thread at those sizes, and more threads were never faster in the measured
// sweeps (2D L=181: 544 and 1024 threads tie; 3D L=32: 512 beats 1024)
template <int DIM, int J, bool SHORT>
__global__ void __launch_bounds__(DIM == 3 ? 512 : 768, 1) k_tiny(StepParams single, const StepParams *table,
                                                  uint32_t warp_mode) {
    extern __shared__ __align__(16) uint32_t tiny_smem[];
    const StepParams p = table ? table[blockIdx.x] : single;
    const TinyGeo g(p.g.L, p.g.N);
    uint32_t *S = tiny_smem;
    uint32_t *Bb = tiny_smem + off_bonds(g);
    uint32_t *Fb = tiny_smem + off_front<DIM>(g);
    uint32_t *sums = tiny_smem + off_sums<DIM>(g);
    __shared__ uint32_t s_seed[2];
    __shared__ uint32_t s_stop[2];   // by update parity: a slow reader never sees the next one
    const uint32_t T = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t nwarps = T >> 5;
    const uint32_t bstride = DIM * g.NW;     // one parity's bond planes
    DevCtl *ctl = p.ctl;
    // warp mode only ever needs two words per lane in 3D (a 2D lattice of at
    // most 64 words has at most 32 rows): the 2D two-word kernel omits it
    constexpr bool kWarpPath = !(DIM == 2 && J == 2);
    const bool wm = kWarpPath && warp_mode != 0u;
    // the words this thread grows: warp mode: lane + 32 j (warp 0 only);
    // otherwise tid + T j
    const bool grower = !wm || warp == 0u;
    const uint32_t gstride = wm ? 32u : T;
    WordNb<DIM> nb[J];
    bool own[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t k = (wm ? lane : tid) + gstride * (uint32_t)j;
        own[j] = grower && k < g.NW;
        nb[j] = word_nb<DIM>(g, own[j] ? k : 0u);
    }

    // the lattice as bit planes; the first update's bonds and seed
    for (uint32_t k = warp; k < g.NW; k += nwarps) {
        const uint32_t r = k / g.W, w = k - r * g.W;
        const uint32_t x = 32u * w + lane;
        const uint32_t bits = __ballot_sync(kFullMask, x < g.L && (p.spins[x + g.L * r] & 1u));
        if (lane == 0) S[k] = bits;
    }
    const unsigned long long t0 = p.t0;
    draw_bonds<DIM, SHORT>(p, g, t0, Bb, warp, nwarps);
    unsigned long long total_C = 0, levels_sum = 0, start_ns = 0;
    uint32_t last_C = 0, last_levels = 0;
    long long E = 0, M = 0;
    if (tid == 0) {
        start_ns = global_ns();
        ctl->st_start_ns = start_ns;
        E = ctl->E;
        M = ctl->M;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
        s_seed[0] = seed_of(p, t0, g.N);
        s_stop[0] = s_stop[1] = 0;
        for (int q = 0; q < 8; ++q) sums[q] = 0u;
    }
    __syncthreads();
    uint32_t Sr[J];   // warp mode: warp 0's rows of spins
#pragma unroll
    for (int j = 0; j < J; ++j) Sr[j] = (wm && own[j]) ? S[nb[j].k] : 0u;

    unsigned long long u = 0;
    while (u < p.n) {
        const uint32_t par = wm ? (uint32_t)(u & 1u) : 0u;
        const unsigned long long t = p.t0 + u;
        if (!wm && u > 0) {
            // this update's bonds (the previous update's readers are past
            // the barrier that closed it)
            draw_bonds<DIM, SHORT>(p, g, t, Bb, warp, nwarps);
            if (tid == 0) s_seed[0] = seed_of(p, t, g.N);
            __syncthreads();
        }
        const uint32_t *B = Bb + par * bstride;
        const uint32_t i0 = s_seed[par];
        uint32_t level = 0, C = 0, anti = 0, up = 0;
        if (kWarpPath && wm && warp == 0u) {
            if constexpr (kWarpPath) warp_update<DIM, J>(g, nb, own, Sr, B, i0, C, anti, up, level);
        } else if (grower) {
            const uint32_t x0 = i0 % g.L, r0 = i0 / g.L;
            const uint32_t seedk = r0 * g.W + (x0 >> 5), seedbit = 1u << (x0 & 31u);
            const uint32_t sig0bit = (S[seedk] & seedbit) ? 1u : 0u;
            WordState ws[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (own[j]) {
                    start_word<DIM>(nb[j], g, S, B, sig0bit, seedk, seedbit, ws[j]);
                    Fb[nb[j].k] = ws[j].F;
                }
            }
            uint32_t cur = 0;
            __syncthreads();
            for (;;) {
                const uint32_t *Fc = Fb + cur * g.NW;
                uint32_t *Fn = Fb + (cur ^ 1u) * g.NW;
                uint32_t any = 0;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if (own[j]) {
                        const uint32_t nw_ = grow_word<DIM>(nb[j], ws[j], Fc);
                        ws[j].V |= nw_;
                        ws[j].F = nw_;
                        Fn[nb[j].k] = nw_;
                        any |= nw_;
                    }
                }
                ++level;
                // the level barrier; it also tells whether the front is empty
                if (!__syncthreads_or(any != 0u)) break;
                cur ^= 1u;
            }
            // flip the cluster
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (own[j]) {
                    S[nb[j].k] ^= ws[j].V;
                    C += __popc(ws[j].V);
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (own[j]) count_word<DIM>(nb[j], S, anti, up);
            C = __reduce_add_sync(kFullMask, C);
            anti = __reduce_add_sync(kFullMask, anti);
            up = __reduce_add_sync(kFullMask, up);
            if (lane == 0) {
                atomicAdd(&sums[0], C);
                atomicAdd(&sums[1], anti);
                atomicAdd(&sums[2], up);
            }
        } else {
            // warp mode helpers: the next update's bonds and seed
            draw_bonds<DIM, SHORT>(p, g, t + 1, Bb + (par ^ 1u) * bstride, warp - 1u, nwarps - 1u);
            if (tid == 32u) s_seed[par ^ 1u] = seed_of(p, t + 1, g.N);
        }
        if (tid == 0 && p.budget_ns)
            s_stop[u & 1u] = global_ns() - start_ns > p.budget_ns ? 1u : 0u;
        __syncthreads();
        if (tid == 0) {
            if (!wm) {
                C = sums[0];
                anti = sums[1];
                up = sums[2];
                sums[0] = sums[1] = sums[2] = 0u;
            }
            E = (long long)DIM * (long long)g.N - 2LL * (long long)anti;
            M = 2LL * (long long)up - (long long)g.N;
            total_C += C;
            last_C = C;
            last_levels = level;
            levels_sum += level;
            if (p.records) {
                wolff_record rec;
                rec.C = C;
                rec.levels = level;
                rec.E_bond = E;
                rec.M = M;
                p.records[u] = rec;
            }
        }
        const bool stop = p.budget_ns && s_stop[u & 1u];
        ++u;
        if (stop) break;
        // the sums are read by thread 0 above before anyone adds again: the
        // next update's adds come after its draw barrier (or, in warp mode,
        // are not made)
    }
    if (wm && warp == 0u) {
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (own[j]) S[nb[j].k] = Sr[j];
    }
    __syncthreads();
    for (uint32_t i = tid; i < g.N; i += T) {
        const uint32_t x = i % g.L, r = i / g.L;
        p.spins[i] = ((S[r * g.W + (x >> 5)] >> (x & 31u)) & 1u) ? 3u : 0u;
    }
    if (tid == 0) {
        ctl->E = E;
        ctl->M = M;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + u;
        ctl->st_updates += u;
        ctl->st_levels_local += levels_sum;
        ctl->st_end_ns = global_ns();
    }
}

constexpr int kAttrDevices = 64;
std::atomic<size_t> g_tiny_smem_set[kAttrDevices][4];

// (only the word-by-word kernels ever need more than the default 48 KB of
// dynamic shared memory: a lattice with rows of at most 16 sites has at most
// 4096 sites)
const void *tiny_kernel(int dim, int J) {
    if (dim == 2)
        return J == 1 ? reinterpret_cast<const void *>(&k_tiny<2, 1, false>)
                      : reinterpret_cast<const void *>(&k_tiny<2, 2, false>);
    return J == 1 ? reinterpret_cast<const void *>(&k_tiny<3, 1, false>)
                  : reinterpret_cast<const void *>(&k_tiny<3, 2, false>);
}

cudaError_t ensure_tiny_smem(int dim, int J, size_t bytes) {
    if (bytes <= 48u * 1024u) return cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrDevices) {
        cudaGetLastError();
        return cudaFuncSetAttribute(tiny_kernel(dim, J),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
    std::atomic<size_t> &cur = g_tiny_smem_set[dev][(dim == 2 ? 0 : 2) + (J == 1 ? 0 : 1)];
    size_t seen = cur.load();
    if (bytes <= seen) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tiny_kernel(dim, J),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    while (seen < bytes && !cur.compare_exchange_weak(seen, bytes)) {
    }
    return cudaSuccess;
}

}  // namespace

uint32_t tiny_words_of(int dim, int L) {
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)L;
    return (uint32_t)(n / (uint64_t)L) * (((uint32_t)L + 31u) / 32u);
}

bool tiny_warp_mode(int dim, int L, int threads) {
    return threads >= 64 && tiny_words_of(dim, L) <= 64u;
}

// words per growing thread (1 or 2; 0 if the CTA cannot run the lattice)
static int tiny_J(int dim, int L, int threads) {
    if (threads < 32 || threads > 1024 || threads % 32) return 0;
    const uint32_t nw = tiny_words_of(dim, L);
    const uint32_t growers = tiny_warp_mode(dim, L, threads) ? 32u : (uint32_t)threads;
    const int J = nw <= growers ? 1 : (nw <= 2u * growers ? 2 : 0);
    if (threads > (dim == 3 ? 512 : 768)) return 0;
    return J;
}

bool tiny_shape_ok(int dim, int L, int threads) { return tiny_J(dim, L, threads) != 0; }

// The default CTA, the fastest of 32..1024 threads on 2D L = 16..181 and 3D
// L = 4..32 at T_c: for lattices of at most 64 words warp 0 and three (2D) or
// seven (3D: more sites per row to draw) drawing warps; else 256 threads up
// to 192 words, 512 up to 1024 words (two words per thread beyond 512: fewer
// warps at the level barrier beat one word per thread), and the fewest that
// hold two words each beyond that.
int tiny_default_threads(int dim, int L) {
    const uint32_t nw = tiny_words_of(dim, L);
    if (nw <= 64u) return dim == 3 ? 256 : 128;
    if (nw <= 192u) return 256;
    if (nw <= 1024u) return 512;
    return (int)(((nw + 1u) / 2u + 31u) / 32u * 32u);
}

size_t tiny_smem_bytes(int dim, int L) {
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)L;
    const TinyGeo g((uint32_t)L, (uint32_t)n);
    return 4u * (size_t)(dim == 2 ? tiny_words<2>(g) : tiny_words<3>(g));
}

cudaError_t launch_tiny(int dim, const StepParams &single, const StepParams *d_table, int njobs,
                        int max_L, int threads, cudaStream_t s) {
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)max_L;
    if (n > kTinyMaxSites || !tiny_shape_ok(dim, max_L, threads) || njobs < 1 ||
        (!d_table && njobs != 1))
        return cudaErrorInvalidValue;
    const bool wm = tiny_warp_mode(dim, max_L, threads);
    const int J = tiny_J(dim, max_L, threads);
    const size_t smem = tiny_smem_bytes(dim, max_L);
    cudaError_t e = ensure_tiny_smem(dim, J, smem);
    if (e != cudaSuccess) return e;
    const uint32_t flag = wm ? 1u : 0u;
    // rows of at most 16 sites (every job's, as the largest's): packed draws
    const bool shortrows = max_L <= 16;
    if (dim == 2) {
        if (shortrows)   k_tiny<2, 1, true><<<njobs, threads, smem, s>>>(single, d_table, flag);
        else if (J == 1) k_tiny<2, 1, false><<<njobs, threads, smem, s>>>(single, d_table, flag);
        else             k_tiny<2, 2, false><<<njobs, threads, smem, s>>>(single, d_table, flag);
    } else {
        if (shortrows && J == 1)
            k_tiny<3, 1, true><<<njobs, threads, smem, s>>>(single, d_table, flag);
        else if (shortrows)
            k_tiny<3, 2, true><<<njobs, threads, smem, s>>>(single, d_table, flag);
        else if (J == 1)
            k_tiny<3, 1, false><<<njobs, threads, smem, s>>>(single, d_table, flag);
        else
            k_tiny<3, 2, false><<<njobs, threads, smem, s>>>(single, d_table, flag);
    }
    return cudaGetLastError();
}

}  // namespace wolff
