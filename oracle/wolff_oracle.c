/*
 * wolff_oracle.c -- plain, slow, single-threaded CPU oracle for the Wolff
 * single-cluster update of the Ising model (Komura & Okabe, "GPU-based
 * single-cluster algorithm for the simulation of the Ising model").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's timed
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only through their outputs.
 *
 * What it computes (section 2 of the paper):
 *   H = -J sum_<ij> S_i S_j on the L^D periodic square (D=2) or simple-cubic
 *   (D=3) lattice.  One update: (i) pick a random site i0; (ii)-(iv) grow the
 *   cluster: every member looks at each nearest neighbour j and adds it when
 *   S_j is parallel to the seed spin and a bond test with probability
 *   p = 1 - exp(-2J/T) succeeds; members are kept in a FIFO list with the
 *   counters ic (members) and in (members already checked), looping while
 *   in < ic; then every member is flipped.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - Randomness.  The paper's linear congruential generator is replaced by the
 *     counter-based Philox4x32-10 of Salmon, Moraes, Dror and Shaw (SC'11),
 *     key = (seed_lo, seed_hi).  Bond (o,d) -- the bond from site o to its
 *     forward neighbour in direction d -- uses lane d of
 *     Philox(ctr = (o, t_lo, t_hi, 0)).  The seed site of update t is
 *     floor(x * N / 2^32) with x = lane 0 of Philox(ctr = (0, t_lo, t_hi, 1)).
 *     The initial spin of site i is -1 when the top bit of lane 0 of
 *     Philox(ctr = (i, 0, 0, 2)) is set, else +1.
 *   - Bond test.  thr = floor(p * 2^32) with p = 1 - exp(-2J/T) evaluated in
 *     IEEE double with the C library's exp; a bond is active when r < thr, so
 *     thr = 2^32 (p = 1) always accepts and thr = 0 never does.
 *   - Small L.  At L = 2 the forward and backward neighbours along an axis are
 *     the same site but the bonds (i,d) and (nb(i,d),d) stay distinct, so the
 *     energy counts D*N directed-forward bonds at every L.
 *   - The cluster is the connected component of the seed in the graph of
 *     active bonds whose both ends carry the seed's spin; the paper leaves the
 *     timing of the flip open, and this file flips the members after growth.
 *   - Measurement ("+ measurement" column of Tables 1-2): the bond sum
 *     E_bond = sum_{i,d} s_i s_{nb(i,d)} and M = sum_i s_i, recounted from
 *     their definitions after every update (physical energy = -J * E_bond).
 *
 * Build: gcc -O2 -std=c99 -shared -fPIC (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Philox4x32-10 (Salmon et al., SC'11, section 3.3 and table 2) ------- */

#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

/* One Philox4x32 round: the two multiplications act on words 0 and 2; the
 * high halves are mixed with words 1 and 3 and the round key.  */
static void orc_philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Ten rounds; the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4],
                       uint32_t out[4])
{
    uint32_t c[4] = { ctr[0], ctr[1], ctr[2], ctr[3] };
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += ORC_PHILOX_W0; k1 += ORC_PHILOX_W1; }
        orc_philox_round(c, k0, k1);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Counter tags: the fourth counter word separates the three uses. */
enum { ORC_TAG_BOND = 0, ORC_TAG_SEED = 1, ORC_TAG_INIT = 2 };

static void orc_draw(uint64_t seed, uint32_t c0, uint64_t t, uint32_t tag,
                     uint32_t out[4])
{
    uint32_t ctr[4] = { c0, (uint32_t)t, (uint32_t)(t >> 32), tag };
    orc_philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, out);
}

/* ---- bond probability (section 2, step (ii)) ------------------------------ */

/* thr = floor(p * 2^32), p = 1 - exp(-2J/T).  Returns 0 for J <= 0 or
 * T = +inf, and 2^32 when p rounds to 1. */
uint64_t orc_bond_threshold(double J, double T)
{
    double p = 1.0 - exp(-2.0 * J / T);
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

/* ---- lattice geometry ---------------------------------------------------- */

/* site i = x + L*y (+ L*L*z).  Neighbour of i one step along axis d with
 * sign +1 or -1, periodic. */
static uint32_t orc_neighbour(int dim, uint32_t L, uint32_t i, int d, int sign)
{
    uint32_t stride = 1;
    for (int k = 0; k < d; ++k) stride *= L;
    uint32_t coord = (i / stride) % L;
    uint32_t moved = sign > 0 ? (coord + 1) % L : (coord + L - 1) % L;
    (void)dim;
    return i + (moved - coord) * stride;   /* unsigned wrap is exact here */
}

static uint32_t orc_sites(int dim, uint32_t L)
{
    uint32_t n = 1;
    for (int k = 0; k < dim; ++k) n *= L;
    return n;
}

/* ---- initial configuration ----------------------------------------------- */

void orc_init(int dim, uint32_t L, uint64_t seed, int8_t *s)
{
    uint32_t n = orc_sites(dim, L);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t r[4];
        orc_draw(seed, i, 0, ORC_TAG_INIT, r);
        s[i] = (r[0] >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

/* ---- observables by definition (section 2, the Hamiltonian) -------------- */

int64_t orc_energy_bond(int dim, uint32_t L, const int8_t *s)
{
    uint32_t n = orc_sites(dim, L);
    int64_t e = 0;
    for (uint32_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d)
            e += (int64_t)s[i] * (int64_t)s[orc_neighbour(dim, L, i, d, +1)];
    return e;
}

int64_t orc_magnetisation(int dim, uint32_t L, const int8_t *s)
{
    uint32_t n = orc_sites(dim, L);
    int64_t m = 0;
    for (uint32_t i = 0; i < n; ++i) m += s[i];
    return m;
}

/* ---- seed site (section 2, step (i)) ------------------------------------- */

uint32_t orc_seed_site(uint64_t seed, uint64_t t, uint32_t n)
{
    uint32_t r[4];
    orc_draw(seed, 0, t, ORC_TAG_SEED, r);
    return (uint32_t)(((uint64_t)r[0] * (uint64_t)n) >> 32);
}

/* Random number of bond (o,d) in update t. */
static uint32_t orc_bond_random(uint64_t seed, uint64_t t, uint32_t o, int d)
{
    uint32_t r[4];
    orc_draw(seed, o, t, ORC_TAG_BOND, r);
    return r[d];
}

/* ---- one cluster (section 2, steps (i)-(iv), ic/in list) ------------------
 *
 * Grows the cluster of update t on configuration s without changing s.
 * member[] must be all zero on entry; on return member[i] = 1 exactly for the
 * cluster's sites and list[0..ic) holds them in the order they were added
 * (breadth-first).  *levels receives the number of breadth-first generations
 * (1 for a lone seed).  Returns ic = |C|. */
uint32_t orc_cluster(int dim, uint32_t L, uint64_t thr, uint64_t seed,
                     uint64_t t, const int8_t *s, uint8_t *member,
                     uint32_t *list, uint32_t *levels)
{
    uint32_t n = orc_sites(dim, L);
    uint32_t i0 = orc_seed_site(seed, t, n);
    int8_t sigma0 = s[i0];
    uint32_t ic = 0, in = 0;
    list[ic++] = i0;
    member[i0] = 1;
    uint32_t generation_end = ic, generations = 1;
    while (in < ic) {
        if (in == generation_end) {          /* next breadth-first generation */
            generation_end = ic;
            ++generations;
        }
        uint32_t i = list[in++];
        for (int d = 0; d < dim; ++d) {
            for (int sign = +1; sign >= -1; sign -= 2) {
                uint32_t j = orc_neighbour(dim, L, i, d, sign);
                uint32_t owner = sign > 0 ? i : j;   /* bond (owner, d) */
                if (member[j] || s[j] != sigma0) continue;
                if ((uint64_t)orc_bond_random(seed, t, owner, d) < thr) {
                    member[j] = 1;
                    list[ic++] = j;
                }
            }
        }
    }
    if (levels) *levels = generations;
    return ic;
}

/* ---- the update loop ----------------------------------------------------- */

typedef struct {
    uint32_t C;        /* |C_t| */
    uint32_t levels;   /* breadth-first generations of the cluster */
    int64_t  E_bond;   /* bond sum after the flip */
    int64_t  M;        /* magnetisation after the flip */
} orc_record;

/* Runs updates t0 .. t0+n-1 on s in place and writes one record per update
 * (rec may be NULL).  Returns 0, or -1 when scratch memory is unavailable. */
int orc_run(int dim, uint32_t L, uint64_t thr, uint64_t seed, uint64_t t0,
            uint64_t n, int8_t *s, orc_record *rec)
{
    uint32_t sites = orc_sites(dim, L);
    uint8_t *member = (uint8_t *)calloc(sites, 1);
    uint32_t *list = (uint32_t *)malloc((size_t)sites * sizeof(uint32_t));
    if (!member || !list) { free(member); free(list); return -1; }
    for (uint64_t u = 0; u < n; ++u) {
        uint64_t t = t0 + u;
        uint32_t levels = 0;
        uint32_t c = orc_cluster(dim, L, thr, seed, t, s, member, list, &levels);
        for (uint32_t k = 0; k < c; ++k) {   /* step (iii): flip the members */
            s[list[k]] = (int8_t)-s[list[k]];
            member[list[k]] = 0;
        }
        if (rec) {
            rec[u].C = c;
            rec[u].levels = levels;
            rec[u].E_bond = orc_energy_bond(dim, L, s);
            rec[u].M = orc_magnetisation(dim, L, s);
        }
    }
    free(member);
    free(list);
    return 0;
}

/* ---- the update loop with the records kept by a local recount -----------
 *
 * The same updates as orc_run (same cluster, same flip), but E_bond and M are
 * counted from their definitions only once, before the first update; after
 * that each record follows from the previous one by recounting, before and
 * after the flip, only the terms the flip can change.  E_bond is a sum over
 * bonds, and a bond's term s_a s_b changes only when one of its ends is
 * flipped, so every bond that does not touch the cluster keeps its term.
 * orc_touching_bonds sums s_a s_b over the 2D bonds at every member i -- its
 * forward bonds (i, nb(i,d,+1)) and the bonds (nb(i,d,-1), i) that end at i
 * -- so a bond with both ends in the cluster is counted twice, before and
 * after alike, and its term (both ends flipped) does not change; a bond with
 * one end in the cluster is counted once.  Hence
 *     E_after = E_before + touching(after) - touching(before),
 *     M_after = M_before + sum over members of (s_after - s_before).
 * This costs O(|C|) per update instead of O(N), so whole runs of the
 * 2^24-site lattices can be replayed record by record. */

static int64_t orc_touching_bonds(int dim, uint32_t L, const int8_t *s,
                                  const uint32_t *list, uint32_t c)
{
    int64_t sum = 0;
    for (uint32_t k = 0; k < c; ++k) {
        uint32_t i = list[k];
        for (int d = 0; d < dim; ++d) {
            sum += (int64_t)s[i] * (int64_t)s[orc_neighbour(dim, L, i, d, +1)];
            sum += (int64_t)s[orc_neighbour(dim, L, i, d, -1)] * (int64_t)s[i];
        }
    }
    return sum;
}

/* em (nullable): on entry E_bond and M of s, which the caller already has
 * (else they are counted here from their definitions); on return those of
 * the final lattice. */
int orc_run_local(int dim, uint32_t L, uint64_t thr, uint64_t seed, uint64_t t0,
                  uint64_t n, int8_t *s, int64_t *em, orc_record *rec)
{
    uint32_t sites = orc_sites(dim, L);
    uint8_t *member = (uint8_t *)calloc(sites, 1);
    uint32_t *list = (uint32_t *)malloc((size_t)sites * sizeof(uint32_t));
    if (!member || !list) { free(member); free(list); return -1; }
    int64_t e = em ? em[0] : orc_energy_bond(dim, L, s);
    int64_t m = em ? em[1] : orc_magnetisation(dim, L, s);
    for (uint64_t u = 0; u < n; ++u) {
        uint64_t t = t0 + u;
        uint32_t levels = 0;
        uint32_t c = orc_cluster(dim, L, thr, seed, t, s, member, list, &levels);
        int64_t before = orc_touching_bonds(dim, L, s, list, c);
        int64_t m_before = 0, m_after = 0;
        for (uint32_t k = 0; k < c; ++k) m_before += s[list[k]];
        for (uint32_t k = 0; k < c; ++k) {   /* step (iii): flip the members */
            s[list[k]] = (int8_t)-s[list[k]];
            member[list[k]] = 0;
        }
        for (uint32_t k = 0; k < c; ++k) m_after += s[list[k]];
        e += orc_touching_bonds(dim, L, s, list, c) - before;
        m += m_after - m_before;
        if (rec) {
            rec[u].C = c;
            rec[u].levels = levels;
            rec[u].E_bond = e;
            rec[u].M = m;
        }
    }
    if (em) { em[0] = e; em[1] = m; }
    free(member);
    free(list);
    return 0;
}

/* ---- exact enumeration of all 2^N states --------------------------------
 *
 * Fills hist[(E_bond + D*N) * (2N+1) + (M + N)] with the number of
 * configurations having that bond sum and magnetisation (the density of
 * states g(E_bond, M)).  The states are visited in binary-reflected Gray-code
 * order, so each step flips one spin and E_bond, M change by the local terms.
 * hist must hold (2*D*N+1)*(2N+1) zeroed entries.  N <= 32. */
int orc_enumerate(int dim, uint32_t L, uint64_t *hist)
{
    uint32_t n = orc_sites(dim, L);
    if (n > 32) return -1;
    int8_t *s = (int8_t *)malloc(n);
    if (!s) return -1;
    for (uint32_t i = 0; i < n; ++i) s[i] = 1;
    int64_t e = orc_energy_bond(dim, L, s);
    int64_t m = n;
    int64_t width = 2 * (int64_t)n + 1, eoff = (int64_t)dim * n;
    hist[(e + eoff) * width + (m + n)] += 1;
    uint64_t total = (uint64_t)1 << n;
    for (uint64_t k = 1; k < total; ++k) {
        uint32_t i = (uint32_t)__builtin_ctzll(k);   /* Gray-code bit to flip */
        int64_t local = 0;
        for (int d = 0; d < dim; ++d) {
            local += s[orc_neighbour(dim, L, i, d, +1)];
            local += s[orc_neighbour(dim, L, i, d, -1)];
        }
        /* flipping s_i changes every bond touching i from s_i s_j to -s_i s_j */
        e -= 2 * (int64_t)s[i] * local;
        m -= 2 * (int64_t)s[i];
        s[i] = (int8_t)-s[i];
        hist[(e + eoff) * width + (m + n)] += 1;
    }
    free(s);
    return 0;
}

/* ==== q-state Potts model (the extension named in section 6) ==============
 *
 * H = -J sum_<ij> delta(c_i, c_j), colours c in {0 .. q-1}.  One Wolff
 * update t: seed site i0 and a new colour c' != c0, both from the seed draw
 * (lane 0 -> site, lane 1 -> c' = (c0 + 1 + floor(x1 (q-1) / 2^32)) mod q);
 * the cluster grows through bonds to neighbours of colour c0 that are active
 * with probability p = 1 - exp(-J/T) (the same bond words as the Ising
 * update); every member then takes colour c'.  With q = 2 this is the Ising
 * update of coupling J/2, colour 1 <-> spin -1.
 * Observables: the satisfied-bond count E_bond = sum_{i,d} delta(c_i, c_nb)
 * (energy -J E_bond) and N0, the number of sites of colour 0.
 * Initial colour of site i: floor(x q / 2^32), x = lane 0 of Philox(i, 0, 0, 2). */

void orc_potts_init(int dim, uint32_t L, uint32_t q, uint64_t seed, int8_t *c)
{
    uint32_t n = orc_sites(dim, L);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t r[4];
        orc_draw(seed, i, 0, ORC_TAG_INIT, r);
        c[i] = (int8_t)(((uint64_t)r[0] * q) >> 32);
    }
}

int64_t orc_potts_energy_bond(int dim, uint32_t L, const int8_t *c)
{
    uint32_t n = orc_sites(dim, L);
    int64_t e = 0;
    for (uint32_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d)
            e += c[i] == c[orc_neighbour(dim, L, i, d, +1)];
    return e;
}

int64_t orc_potts_count0(int dim, uint32_t L, const int8_t *c)
{
    uint32_t n = orc_sites(dim, L);
    int64_t k = 0;
    for (uint32_t i = 0; i < n; ++i) k += c[i] == 0;
    return k;
}

/* Cluster of Potts update t on c (c unchanged); member[] zero on entry.
 * Writes the new colour to *new_colour.  Returns |C|. */
uint32_t orc_potts_cluster(int dim, uint32_t L, uint32_t q, uint64_t thr, uint64_t seed,
                           uint64_t t, const int8_t *c, uint8_t *member, uint32_t *list,
                           uint32_t *levels, int *new_colour)
{
    uint32_t n = orc_sites(dim, L);
    uint32_t r[4];
    orc_draw(seed, 0, t, ORC_TAG_SEED, r);
    uint32_t i0 = (uint32_t)(((uint64_t)r[0] * n) >> 32);
    int c0 = c[i0];
    *new_colour = (int)((c0 + 1 + (((uint64_t)r[1] * (q - 1)) >> 32)) % q);
    uint32_t ic = 0, in = 0;
    list[ic++] = i0;
    member[i0] = 1;
    uint32_t generation_end = ic, generations = 1;
    while (in < ic) {
        if (in == generation_end) {
            generation_end = ic;
            ++generations;
        }
        uint32_t i = list[in++];
        for (int d = 0; d < dim; ++d) {
            for (int sign = +1; sign >= -1; sign -= 2) {
                uint32_t j = orc_neighbour(dim, L, i, d, sign);
                uint32_t owner = sign > 0 ? i : j;
                if (member[j] || c[j] != c0) continue;
                if ((uint64_t)orc_bond_random(seed, t, owner, d) < thr) {
                    member[j] = 1;
                    list[ic++] = j;
                }
            }
        }
    }
    if (levels) *levels = generations;
    return ic;
}

/* Potts updates t0 .. t0+n-1 on c in place; records (nullable) hold |C|,
 * levels, E_bond (satisfied bonds) and N0 in the M field. */
int orc_potts_run(int dim, uint32_t L, uint32_t q, uint64_t thr, uint64_t seed, uint64_t t0,
                  uint64_t n, int8_t *c, orc_record *rec)
{
    uint32_t sites = orc_sites(dim, L);
    uint8_t *member = (uint8_t *)calloc(sites, 1);
    uint32_t *list = (uint32_t *)malloc((size_t)sites * sizeof(uint32_t));
    if (!member || !list || q < 2) { free(member); free(list); return -1; }
    for (uint64_t u = 0; u < n; ++u) {
        uint32_t levels = 0;
        int nc = 0;
        uint32_t k = orc_potts_cluster(dim, L, q, thr, seed, t0 + u, c, member, list, &levels,
                                       &nc);
        for (uint32_t m = 0; m < k; ++m) {
            c[list[m]] = (int8_t)nc;
            member[list[m]] = 0;
        }
        if (rec) {
            rec[u].C = k;
            rec[u].levels = levels;
            rec[u].E_bond = orc_potts_energy_bond(dim, L, c);
            rec[u].M = orc_potts_count0(dim, L, c);
        }
    }
    free(member);
    free(list);
    return 0;
}

/* Exact enumeration of all q^N colourings (N small): hist[E_bond * (N+1) + N0]
 * counts, E_bond in 0..D*N.  Colourings are visited as base-q numbers. */
int orc_potts_enumerate(int dim, uint32_t L, uint32_t q, uint64_t *hist)
{
    uint32_t n = orc_sites(dim, L);
    double states = 1.0;
    for (uint32_t i = 0; i < n; ++i) states *= q;
    if (states > 1.0e9) return -1;
    int8_t *c = (int8_t *)calloc(n, 1);
    if (!c) return -1;
    uint64_t total = (uint64_t)states;
    for (uint64_t k = 0; k < total; ++k) {
        int64_t e = orc_potts_energy_bond(dim, L, c);
        int64_t z = orc_potts_count0(dim, L, c);
        hist[e * (n + 1) + z] += 1;
        for (uint32_t i = 0; i < n; ++i) {   /* next base-q colouring */
            if (++c[i] < (int8_t)q) break;
            c[i] = 0;
        }
    }
    free(c);
    return 0;
}

uint64_t orc_potts_threshold(double J, double T)
{
    double p = 1.0 - exp(-J / T);
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

/* ---- XY model (section 6 names it as the next extension) -----------------
 *
 * H = -J sum_<ij> cos(theta_i - theta_j).  Wolff's embedded-cluster update
 * (Wolff, PRL 62 (1989) 361): draw a unit vector r at angle phi and a seed
 * site; a bond <ij> is active with probability
 *     p_ij = 1 - exp(-2K (r.s_i)(r.s_j))  when (r.s_i)(r.s_j) > 0, else 0,
 * K = J/T, judged on the pre-update spins; the cluster is the seed's
 * connected component of active bonds, and every member is reflected in the
 * line perpendicular to r: theta -> pi + 2 phi - theta.
 *
 * Readings (exact integer arithmetic, so that CPU and GPU agree bit for bit):
 *   - Angles are integers in units of 2 pi / 65536.  With angle_bits b
 *     (1..15) spins are multiples of 2^(16-b) and phi a multiple of
 *     2^(15-b), so the reflection 32768 + 2 phi - theta (mod 65536) stays on
 *     the grid; b = 15 is the production resolution, small b gives a
 *     2^b-state clock model whose Boltzmann averages can be enumerated.
 *   - cos is the fixed-point table I[k] = round(cos(pi k / 32768) 2^30),
 *     k = 0..16384 (C library cos in double), extended by symmetry.  The
 *     projection r.s_i is I(theta_i - phi); E_fix = sum_{i,d} I(theta_i -
 *     theta_nb(i,d)) (energy -J E_fix 2^-30); Mx = sum I(theta_i),
 *     My = sum I(theta_i - 16384).
 *   - p_ij: y = (2K 2^-60) * (double)(I_i I_j) and p = 1 - e^-y, with e^-y
 *     computed by Cody-Waite range reduction (y = k ln2 + r) and the Taylor
 *     series of e^-r to degree 16 (Cody & Waite, Software Manual for the
 *     Elementary Functions, 1980) in IEEE double basic operations in a fixed
 *     order (no contraction), so that any platform following the same steps
 *     gets the same double; thr = floor(p 2^32) and the bond is active when
 *     its random word is below thr.
 *   - Randomness: the seed site as in the Ising update (lane 0 of the seed
 *     draw), phi from lane 1 of the same draw, the bond words as in the Ising
 *     update; initial angle of site i from lane 0 of Philox(i, 0, 0, 2). */

typedef struct {
    uint32_t C;
    uint32_t levels;
    int64_t  E;    /* fixed-point bond sum E_fix after the flip */
    int64_t  Mx;   /* fixed-point magnetisation after the flip */
    int64_t  My;
} orc_xy_record;

#define ORC_XY_PI 3.141592653589793

void orc_xy_table(int32_t *tab)
{
    for (int k = 0; k <= 16384; ++k)
        tab[k] = (int32_t)llround(cos(ORC_XY_PI * (double)k / 32768.0) * 1073741824.0);
}

/* cos of angle a (units 2 pi / 65536) from the quarter-wave table. */
static int32_t orc_xy_cos(const int32_t *tab, uint32_t a)
{
    a &= 0xFFFFu;
    uint32_t q = a >> 14, r = a & 0x3FFFu;
    if (q == 0) return tab[r];
    if (q == 1) return -tab[16384 - r];
    if (q == 2) return -tab[r];
    return tab[16384 - r];
}

int32_t orc_xy_cos_at(uint32_t a)
{
    static int32_t tab[16385];
    static int ready = 0;
    if (!ready) { orc_xy_table(tab); ready = 1; }
    return orc_xy_cos(tab, a);
}

/* e^-y for y >= 0 (see the readings above). */
double orc_xy_exp_neg(double y)
{
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_hi = 0x1.62e42feep-1;      /* ln 2 to 32 significant bits */
    const double ln2_lo = 0x1.a39ef35793c76p-33; /* ln 2 - ln2_hi */
    if (!(y < 1000.0)) return 0.0;
    double coef[17];
    coef[0] = 1.0;
    for (int n = 1; n <= 16; ++n) coef[n] = coef[n - 1] / (double)n;
    double t = y * inv_ln2;
    double kd = floor(t + 0.5);
    double r = (y - kd * ln2_hi) - kd * ln2_lo;
    double m = -r;
    double s = coef[16];
    for (int n = 15; n >= 0; --n) s = s * m + coef[n];
    return ldexp(s, -(int)kd);
}

/* 2K 2^-60, the factor that turns a product of two projections into y. */
double orc_xy_coupling(double J, double T)
{
    return ldexp(2.0 * J / T, -60);
}

uint64_t orc_xy_threshold(int64_t prod, double kk)
{
    if (prod <= 0) return 0;
    double y = kk * (double)prod;
    double p = 1.0 - orc_xy_exp_neg(y);
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

void orc_xy_init(int dim, uint32_t L, int bits, uint64_t seed, uint16_t *theta)
{
    uint32_t n = orc_sites(dim, L);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t r[4];
        orc_draw(seed, i, 0, ORC_TAG_INIT, r);
        theta[i] = (uint16_t)((r[0] >> (32 - bits)) << (16 - bits));
    }
}

void orc_xy_observables(int dim, uint32_t L, const uint16_t *theta, int64_t out[3])
{
    uint32_t n = orc_sites(dim, L);
    int64_t e = 0, mx = 0, my = 0;
    for (uint32_t i = 0; i < n; ++i) {
        for (int d = 0; d < dim; ++d)
            e += orc_xy_cos_at((uint32_t)theta[i] - theta[orc_neighbour(dim, L, i, d, +1)]);
        mx += orc_xy_cos_at(theta[i]);
        my += orc_xy_cos_at((uint32_t)theta[i] + 65536u - 16384u);
    }
    out[0] = e;
    out[1] = mx;
    out[2] = my;
}

/* Reflection angle of update t on the grid of angle_bits b. */
uint32_t orc_xy_phi(uint64_t seed, uint64_t t, int bits)
{
    uint32_t r[4];
    orc_draw(seed, 0, t, ORC_TAG_SEED, r);
    return (r[1] >> (32 - (bits + 1))) << (15 - bits);
}

/* Cluster of XY update t on theta (unchanged); member[] zero on entry.
 * Writes phi.  Returns |C|. */
uint32_t orc_xy_cluster(int dim, uint32_t L, int bits, double kk, uint64_t seed, uint64_t t,
                        const uint16_t *theta, uint8_t *member, uint32_t *list, uint32_t *levels,
                        uint32_t *phi_out)
{
    uint32_t n = orc_sites(dim, L);
    uint32_t r[4];
    orc_draw(seed, 0, t, ORC_TAG_SEED, r);
    uint32_t i0 = (uint32_t)(((uint64_t)r[0] * n) >> 32);
    uint32_t phi = orc_xy_phi(seed, t, bits);
    if (phi_out) *phi_out = phi;
    uint32_t ic = 0, in = 0;
    list[ic++] = i0;
    member[i0] = 1;
    uint32_t generation_end = ic, generations = 1;
    while (in < ic) {
        if (in == generation_end) {
            generation_end = ic;
            ++generations;
        }
        uint32_t i = list[in++];
        int64_t si = orc_xy_cos_at((uint32_t)theta[i] + 65536u - phi);
        for (int d = 0; d < dim; ++d) {
            for (int sign = +1; sign >= -1; sign -= 2) {
                uint32_t j = orc_neighbour(dim, L, i, d, sign);
                uint32_t owner = sign > 0 ? i : j;
                if (member[j]) continue;
                int64_t sj = orc_xy_cos_at((uint32_t)theta[j] + 65536u - phi);
                uint64_t thr = orc_xy_threshold(si * sj, kk);
                if ((uint64_t)orc_bond_random(seed, t, owner, d) < thr) {
                    member[j] = 1;
                    list[ic++] = j;
                }
            }
        }
    }
    if (levels) *levels = generations;
    return ic;
}

/* XY updates t0 .. t0+n-1 on theta in place; records (nullable) recounted
 * from their definitions after every update. */
int orc_xy_run(int dim, uint32_t L, int bits, double kk, uint64_t seed, uint64_t t0, uint64_t n,
               uint16_t *theta, orc_xy_record *rec)
{
    uint32_t sites = orc_sites(dim, L);
    if (bits < 1 || bits > 15) return -1;
    uint8_t *member = (uint8_t *)calloc(sites, 1);
    uint32_t *list = (uint32_t *)malloc((size_t)sites * sizeof(uint32_t));
    if (!member || !list) { free(member); free(list); return -1; }
    for (uint64_t u = 0; u < n; ++u) {
        uint32_t levels = 0, phi = 0;
        uint32_t k = orc_xy_cluster(dim, L, bits, kk, seed, t0 + u, theta, member, list, &levels,
                                    &phi);
        for (uint32_t m = 0; m < k; ++m) {
            uint32_t i = list[m];
            theta[i] = (uint16_t)((32768u + 2u * phi - theta[i]) & 0xFFFFu);
            member[i] = 0;
        }
        if (rec) {
            int64_t obs[3];
            orc_xy_observables(dim, L, theta, obs);
            rec[u].C = k;
            rec[u].levels = levels;
            rec[u].E = obs[0];
            rec[u].Mx = obs[1];
            rec[u].My = obs[2];
        }
    }
    free(member);
    free(list);
    return 0;
}

/* XY updates as orc_xy_run, with the records kept by a local recount (the
 * argument of orc_run_local): E, Mx and My are counted from their definitions
 * before the first update; after that only the terms of the bonds and sites
 * a reflection changes are recounted, before and after it.  Each bond
 * touching a member is visited from each of its member ends, in the
 * orientation of the definition (the forward bond (i, nb(i,d,+1)) as
 * I(theta_i - theta_nb), the bond ending at i as I(theta_prev - theta_i)).
 * A bond inside the cluster is visited twice, before and after alike, and
 * keeps its term: the reflection theta -> c - theta maps theta_a - theta_b to
 * theta_b - theta_a, and I is even (the table is extended by symmetry).  A
 * bond with one end in the cluster is visited once. */
static int64_t orc_xy_touching(int dim, uint32_t L, const uint16_t *theta, const uint32_t *list,
                               uint32_t c)
{
    int64_t sum = 0;
    for (uint32_t k = 0; k < c; ++k) {
        uint32_t i = list[k];
        for (int d = 0; d < dim; ++d) {
            sum += orc_xy_cos_at((uint32_t)theta[i] - theta[orc_neighbour(dim, L, i, d, +1)]);
            sum += orc_xy_cos_at((uint32_t)theta[orc_neighbour(dim, L, i, d, -1)] - theta[i]);
        }
    }
    return sum;
}

int orc_xy_run_local(int dim, uint32_t L, int bits, double kk, uint64_t seed, uint64_t t0,
                     uint64_t n, uint16_t *theta, orc_xy_record *rec)
{
    uint32_t sites = orc_sites(dim, L);
    if (bits < 1 || bits > 15) return -1;
    uint8_t *member = (uint8_t *)calloc(sites, 1);
    uint32_t *list = (uint32_t *)malloc((size_t)sites * sizeof(uint32_t));
    if (!member || !list) { free(member); free(list); return -1; }
    int64_t obs[3];
    orc_xy_observables(dim, L, theta, obs);
    for (uint64_t u = 0; u < n; ++u) {
        uint32_t levels = 0, phi = 0;
        uint32_t k = orc_xy_cluster(dim, L, bits, kk, seed, t0 + u, theta, member, list, &levels,
                                    &phi);
        int64_t e_before = orc_xy_touching(dim, L, theta, list, k);
        int64_t mx_before = 0, my_before = 0, mx_after = 0, my_after = 0;
        for (uint32_t m = 0; m < k; ++m) {
            mx_before += orc_xy_cos_at(theta[list[m]]);
            my_before += orc_xy_cos_at((uint32_t)theta[list[m]] + 65536u - 16384u);
        }
        for (uint32_t m = 0; m < k; ++m) {
            uint32_t i = list[m];
            theta[i] = (uint16_t)((32768u + 2u * phi - theta[i]) & 0xFFFFu);
            member[i] = 0;
        }
        for (uint32_t m = 0; m < k; ++m) {
            mx_after += orc_xy_cos_at(theta[list[m]]);
            my_after += orc_xy_cos_at((uint32_t)theta[list[m]] + 65536u - 16384u);
        }
        obs[0] += orc_xy_touching(dim, L, theta, list, k) - e_before;
        obs[1] += mx_after - mx_before;
        obs[2] += my_after - my_before;
        if (rec) {
            rec[u].C = k;
            rec[u].levels = levels;
            rec[u].E = obs[0];
            rec[u].Mx = obs[1];
            rec[u].My = obs[2];
        }
    }
    free(member);
    free(list);
    return 0;
}
