/*
 * ea_oracle.c -- plain CPU oracle for the 3D +-J Edwards-Anderson ageing
 * simulation of Manssen & Hartmann, "Ageing at the Spin-Glass/Ferromagnet
 * Transition: Monte Carlo Simulation using GPUs" (arXiv 1411.5512).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is a per-site loop over int8 spins S = +-1 and int8 couplings
 * J = +-1, stored as S[a][i] (replica a in {0,1}) and J[d][i] (direction d in
 * {x,y,z}), with the site index i = x + L*(y + L*z).  The coupling J[d][i]
 * is the bond between site i and its forward neighbour i + e_d (periodic).
 *
 * What is computed, and where the paper defines it:
 *   - Hamiltonian H = -sum_<ij> J_ij S_i S_j, bimodal J, periodic lattice
 *     (Sec. II, Eq. 1).  p_neg here is the fraction of NEGATIVE bonds, i.e.
 *     1 - p in the paper's P(J) = p delta(J-1) + (1-p) delta(J+1).
 *   - Random start ("quench from infinite temperature", Sec. II).
 *   - Metropolis acceptance p = min(1, exp(-(2/T) sum_j J_ij S_i S_j))
 *     (Sec. III, Eq. 9), and the heat-bath rule 1/(1+exp(dE/T)) as a variant.
 *   - Checkerboard schedule: one sweep = update all sites of one colour, then
 *     all sites of the other (Sec. III).  Replica 1 runs the opposite colour
 *     order to replica 0, as the interlaced layout of Fig. 1 implies.
 *
 * Random numbers: the paper's xorshift1024 generator is replaced by the
 * counter-based Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11), written here from that
 * publication.  The mapping from (seed, sample, replica, word-site, sweep) to
 * the 64-bit uniform numbers that decide the flips is a definition of this
 * library (the paper's generator cannot be reproduced); it is restated in
 * full beside draw64 below, the one function that cuts every draw.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_BAD_ARG (-1)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 3: Philox-4x32 with multipliers 0xD2511F53 and */
/* 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85, 10 rounds).   */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Counter word 2 carries a stream tag in its top two bits. */
#define STREAM_COUPLINGS 0u
#define STREAM_SPINS 1u
#define STREAM_HEAT 2u

/* ------------------------------------------------------------------------ */
/* Lattice geometry of the random-number mapping.                           */
/*                                                                          */
/* A "word-site" groups up to 32 lattice sites of one sample that are drawn */
/* from the same Philox calls (see metro_draw and heat_draw).  The        */
/* lattice is cut into kx*ky*kz equal blocks, each of even side, and the    */
/* word-site (x', y', z') of the sub-lattice of side (L/kx, L/ky, L/kz)     */
/* gathers the sites at the same relative position in every block (the     */
/* multi-part packing of Sec. III, extended to three axes).  Rule, fixed by */
/* L alone: with h = L/2 and p2 the largest power of two dividing h,        */
/*   kz = min(32, p2), ky = min(32/kz, p2), kx = min(32/(kz*ky), p2).       */
/* ------------------------------------------------------------------------ */
int ora_geometry(int L, int out[6])
{
    if (L < 2 || L > 1024 || (L & 1))
        return ORA_BAD_ARG;
    int h = L / 2;
    int p2 = h & (-h);
    int kz = p2 < 32 ? p2 : 32;
    int ky = (32 / kz) < p2 ? (32 / kz) : p2;
    int kx = (32 / (kz * ky)) < p2 ? (32 / (kz * ky)) : p2;
    out[0] = kx;
    out[1] = ky;
    out[2] = kz;
    out[3] = L / kx;
    out[4] = L / ky;
    out[5] = L / kz;
    return ORA_OK;
}

/* Word-site index and bit (lane) of site (x, y, z). */
static void site_to_word(int L, int x, int y, int z, uint32_t *widx, int *lane)
{
    int g[6];
    ora_geometry(L, g);
    int kx = g[0], ky = g[1];
    int Lx = g[3], Ly = g[4], Lz = g[5];
    int xw = x % Lx, yw = y % Ly, zw = z % Lz;
    int bx = x / Lx, by = y / Ly, bz = z / Lz;
    *widx = (uint32_t)(xw + Lx * (yw + Ly * zw));
    *lane = bx + kx * (by + ky * bz);
}

int ora_site_to_word(int L, int x, int y, int z, uint32_t *widx, int *lane)
{
    if (L < 2 || L > 1024 || (L & 1) || x < 0 || y < 0 || z < 0 || x >= L || y >= L || z >= L)
        return ORA_BAD_ARG;
    site_to_word(L, x, y, z, widx, lane);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Flip probabilities, one per energy change dE = 4k - 12, k = 0..6, as     */
/* 64-bit fixed point: thr[k] = floor(2^64 P(dE)), always[k] when P == 1.    */
/*   rule 0, Metropolis (Eq. 9):  P = min(1, exp(-dE/T))                    */
/*   rule 1, heat bath:           P = 1 / (1 + exp(dE/T))                   */
/* T = 0 and T = +inf are the limits of P.  The half-step realises these    */
/* probabilities class by class (geometric gaps below; the heat bath's      */
/* dE = 0 by a coin); here always[k] marks the outright Metropolis classes  */
/* and thr[k] == 0 a class that never flips.                                */
/* ------------------------------------------------------------------------ */
int ora_thresholds(double T, int rule, uint64_t thr[7], uint8_t always[7])
{
    if (!(T >= 0.0) || (rule != 0 && rule != 1))
        return ORA_BAD_ARG; /* also rejects NaN */
    for (int k = 0; k < 7; k++) {
        int dE = 4 * k - 12;
        double P;
        if (rule == 0) {
            if (dE <= 0)
                P = 1.0;
            else if (T == 0.0)
                P = 0.0;
            else
                P = exp(-(double)dE / T);
        } else {
            if (T == 0.0)
                P = dE < 0 ? 1.0 : (dE == 0 ? 0.5 : 0.0);
            else
                P = 1.0 / (1.0 + exp((double)dE / T));
        }
        if (P >= 1.0) {
            always[k] = 1;
            thr[k] = 0;
        } else {
            always[k] = 0;
            thr[k] = (uint64_t)floor(ldexp(P, 64));
        }
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Initial state.                                                           */
/* Couplings: J[d][i] = -1 when output d of Philox(ctr = (i, 0, 0, s)) is   */
/* below floor(p_neg * 2^32) (2^32 for p_neg = 1), else +1; i.i.d. per bond. */
/* Spins: S[a][i] = -1 when the top bit of output a of                      */
/* Philox(ctr = (i, 0, 1 << 30, s)) is set, else +1; uniform random start.   */
/* ------------------------------------------------------------------------ */
int ora_init_couplings(int L, double p_neg, uint64_t seed, uint32_t s, int8_t *J)
{
    if (L < 2 || L > 1024 || (L & 1) || !(p_neg >= 0.0 && p_neg <= 1.0))
        return ORA_BAD_ARG;
    uint64_t thr = p_neg >= 1.0 ? ((uint64_t)1 << 32) : (uint64_t)floor(ldexp(p_neg, 32));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t N = (int64_t)L * L * L;
    for (int64_t i = 0; i < N; i++) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, STREAM_COUPLINGS << 30, s};
        uint32_t out[4];
        ora_philox4x32_10(ctr, key, out);
        for (int d = 0; d < 3; d++)
            J[d * N + i] = ((uint64_t)out[d] < thr) ? (int8_t)-1 : (int8_t)1;
    }
    return ORA_OK;
}

/* Couplings with an exact count: K = floor(p_neg * 3N + 1/2) of the 3N bonds
   are negative, the K-subset drawn uniformly.  Bond b = d N + i gets the
   64-bit key (out0 << 32) | out1 of Philox(ctr = (i, 1 + d, 0, s)); the
   negative bonds are the first K in the order of (key, b). */
struct bond_key {
    uint64_t key;
    uint32_t b;
};

static int bond_key_cmp(const void *pa, const void *pb)
{
    const struct bond_key *a = (const struct bond_key *)pa, *b = (const struct bond_key *)pb;
    if (a->key != b->key)
        return a->key < b->key ? -1 : 1;
    return a->b < b->b ? -1 : (a->b > b->b ? 1 : 0);
}

int ora_init_couplings_exact(int L, double p_neg, uint64_t seed, uint32_t s, int8_t *J)
{
    if (L < 2 || L > 1024 || (L & 1) || !(p_neg >= 0.0 && p_neg <= 1.0))
        return ORA_BAD_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t N = (int64_t)L * L * L;
    uint64_t K = (uint64_t)floor(p_neg * 3.0 * (double)N + 0.5);
    struct bond_key *keys = (struct bond_key *)malloc((size_t)(3 * N) * sizeof(struct bond_key));
    if (!keys)
        return ORA_BAD_ARG;
    for (int d = 0; d < 3; d++)
        for (int64_t i = 0; i < N; i++) {
            uint32_t ctr[4] = {(uint32_t)i, 1u + (uint32_t)d, STREAM_COUPLINGS << 30, s};
            uint32_t out[4];
            ora_philox4x32_10(ctr, key, out);
            keys[d * N + i].key = ((uint64_t)out[0] << 32) | out[1];
            keys[d * N + i].b = (uint32_t)(d * N + i);
        }
    qsort(keys, (size_t)(3 * N), sizeof(struct bond_key), bond_key_cmp);
    for (int64_t b = 0; b < 3 * N; b++)
        J[b] = 1;
    for (uint64_t r = 0; r < K; r++)
        J[keys[r].b] = -1;
    free(keys);
    return ORA_OK;
}

int ora_init_spins(int L, uint64_t seed, uint32_t s, int8_t *S)
{
    if (L < 2 || L > 1024 || (L & 1))
        return ORA_BAD_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t N = (int64_t)L * L * L;
    for (int64_t i = 0; i < N; i++) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, STREAM_SPINS << 30, s};
        uint32_t out[4];
        ora_philox4x32_10(ctr, key, out);
        for (int a = 0; a < 2; a++)
            S[a * N + i] = (out[a] >> 31) ? (int8_t)-1 : (int8_t)1;
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Acceptance by geometric gaps (both rules).                               */
/*                                                                          */
/* The sites of one word-site that share a class must each flip             */
/* independently with the same probability p (for Metropolis, class u =    */
/* (12 - dE) / 4 unsatisfied bonds with dE > 0 has p_u = exp(-dE/T), Eq. 9). */
/* Taken in increasing lane order they form a Bernoulli(p) sequence, and    */
/* the number G of failures before the first success is geometric:          */
/* P(G >= g) = (1 - p)^g.  One 64-bit uniform V decides the first success   */
/* among n remaining sites: none if V >= C[n], else the site of rank        */
/* G = min{g : V < C[g+1]}, with                                            */
/*   C[g] = floor(2^64 (1 - (1 - p)^g)),  computed as                       */
/*   floor(ldexp(-expm1(g * log1p(-p)), 64)), clamped to 2^64 - 1.           */
/* The sites after a success start a fresh gap with the next draw.          */
/* ------------------------------------------------------------------------ */
int ora_geo_table(double p, uint64_t C[33])
{
    if (!(p > 0.0 && p < 1.0))
        return ORA_BAD_ARG;
    C[0] = 0;
    for (int g = 1; g <= 32; g++) {
        double q = -expm1((double)g * log1p(-p)); /* 1 - (1 - p)^g */
        double v = ldexp(q, 64);
        C[g] = (v >= 18446744073709551615.0) ? UINT64_MAX : (uint64_t)floor(v);
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* The draws.  Every 64-bit uniform V that decides flips, and the heat      */
/* bath's coin word, is cut from Philox4x32-10 calls with key               */
/* (lo32(seed), hi32(seed)) and counter                                     */
/*   (widx, lo32(t), stream << 30 | (bits 32..47 of t) << 12 | a << 11 | call, s) */
/* where widx = x' + Lx (y' + Ly z') is a word-site of the Lx x Ly x Lz word */
/* lattice, a the replica updated there, t the sweep and s the sample (or   */
/* the sample divided by G).  Stream 3 is Metropolis, stream 2 the heat     */
/* bath.  The assignment of outputs to draws is a definition of this        */
/* library (the paper's generator cannot be reproduced); draw64 below is    */
/* the whole of it:                                                          */
/*                                                                          */
/* Metropolis, class u in {0, 1, 2}, draw d:                                */
/*   d = 0: the leading bits come from the main call of the word-site's     */
/*     quad (x' even, x' + 1) x (z' even, z' + 1): call 0 at the quad's      */
/*     first word-site (x' even, y', z' even), with the replica updated      */
/*     there.  Its output k = (x' mod 2) + 2 (z' mod 2) belongs to this      */
/*     word-site: bits 31..20 lead class 2 (V bits 63..52), bits 19..10     */
/*     class 1 (63..54), bits 9..0 class 0 (63..54).  The rest of V comes   */
/*     from the word-site's own extension calls: call 64 gives              */
/*     (out0:out1) >> 12 to class 2 (V bits 51..0) and (out2:out3) >> 10 to */
/*     class 1 (53..0); call 65 gives (out0:out1) >> 10 to class 0 (53..0). */
/*   d >= 1: (out[2e]:out[2e+1]) of call 1 + u + 3 ((d-1) div 2),            */
/*     e = (d - 1) mod 2.                                                   */
/* Heat bath, class u != 3, pair index j = min(u, 6 - u):                   */
/*   d = 0: V bits 63..48 are bits 31..16 (u < 3) or 15..0 (u > 3) of       */
/*     output 3 - j of call 0; V bits 47..0 are (out0:out1) >> 16 (u < 3)   */
/*     or (out2:out3) >> 16 (u > 3) of call 128 + (2 - j).                  */
/*   d >= 1: (out[2e]:out[2e+1]) of call 1 + u + 7 ((d-1) div 2),            */
/*     e = (d - 1) mod 2 (calls below 128 for d <= 32).                     */
/*   The coin word of class 3 (dE = 0) is output 0 of call 0: bit b decides  */
/*   lane b.                                                                */
/* Why the Metropolis leads are shared per quad: at low T nearly every word  */
/* is settled by its leading bits alone, so a quarter of a Philox call per  */
/* word-site decides it; the rest of a draw is needed only when the leading */
/* bits fall at or below the table.                                          */
/* ------------------------------------------------------------------------ */
#define STREAM_METROPOLIS 3u

static void flip_call(uint32_t stream, uint32_t widx, uint64_t seed, uint32_t s, int a,
                      uint64_t t, int call, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {widx, (uint32_t)t,
                       (stream << 30) | ((uint32_t)((t >> 32) & 0xFFFFu) << 12) |
                           ((uint32_t)a << 11) | (uint32_t)call,
                       s};
    ora_philox4x32_10(ctr, key, out);
}

static uint64_t join64(uint32_t hi, uint32_t lo)
{
    return ((uint64_t)hi << 32) | (uint64_t)lo;
}

/* Draw d of class u at word-site (xw, yw, zw), replica a, sweep t. */
static uint64_t draw64(int rule, int Lx, int Ly, int xw, int yw, int zw, uint64_t seed,
                       uint32_t s, int a, uint64_t t, int u, int d)
{
    uint32_t widx = (uint32_t)(xw + Lx * (yw + Ly * zw));
    uint32_t out[4];
    if (rule == 0) {
        if (d >= 1) {
            int e = (d - 1) % 2;
            flip_call(STREAM_METROPOLIS, widx, seed, s, a, t, 1 + u + 3 * ((d - 1) / 2), out);
            return join64(out[2 * e], out[2 * e + 1]);
        }
        int ox = xw & 1, oz = zw & 1;
        uint32_t widx_q = (uint32_t)((xw - ox) + Lx * (yw + Ly * (zw - oz)));
        flip_call(STREAM_METROPOLIS, widx_q, seed, s, a ^ ox ^ oz, t, 0, out);
        uint32_t lead = out[ox + 2 * oz];
        if (u == 2) {
            flip_call(STREAM_METROPOLIS, widx, seed, s, a, t, 64, out);
            return ((uint64_t)(lead >> 20) << 52) | (join64(out[0], out[1]) >> 12);
        }
        if (u == 1) {
            flip_call(STREAM_METROPOLIS, widx, seed, s, a, t, 64, out);
            return ((uint64_t)((lead >> 10) & 0x3FFu) << 54) | (join64(out[2], out[3]) >> 10);
        }
        flip_call(STREAM_METROPOLIS, widx, seed, s, a, t, 65, out);
        return ((uint64_t)(lead & 0x3FFu) << 54) | (join64(out[0], out[1]) >> 10);
    }
    if (d >= 1) {
        int e = (d - 1) % 2;
        flip_call(STREAM_HEAT, widx, seed, s, a, t, 1 + u + 7 * ((d - 1) / 2), out);
        return join64(out[2 * e], out[2 * e + 1]);
    }
    int pair = u < 3 ? u : 6 - u;
    flip_call(STREAM_HEAT, widx, seed, s, a, t, 0, out);
    uint32_t word = out[3 - pair];
    uint64_t lead = u < 3 ? (word >> 16) : (word & 0xFFFFu);
    flip_call(STREAM_HEAT, widx, seed, s, a, t, 128 + (2 - pair), out);
    uint64_t low = u < 3 ? (join64(out[0], out[1]) >> 16) : (join64(out[2], out[3]) >> 16);
    return (lead << 48) | low;
}

/* The heat bath's coin word of a word-site. */
static uint32_t coin_word(int Lx, int Ly, int xw, int yw, int zw, uint64_t seed, uint32_t s,
                          int a, uint64_t t)
{
    uint32_t out[4];
    flip_call(STREAM_HEAT, (uint32_t)(xw + Lx * (yw + Ly * zw)), seed, s, a, t, 0, out);
    return out[0];
}

/* The lanes of the mask `lanes` (ranked in increasing lane order) that the
   geometric gaps of table C select, with the draws d = 0, 1, ... of class u. */
static uint32_t gap_select(const uint64_t C[33], uint32_t lanes, int rule, int Lx, int Ly,
                           int xw, int yw, int zw, uint64_t seed, uint32_t s, int a,
                           uint64_t t, int u)
{
    int list[32], n = 0;
    for (int b = 0; b < 32; b++)
        if ((lanes >> b) & 1u)
            list[n++] = b;
    uint32_t selected = 0;
    int start = 0, d = 0;
    while (n - start > 0) {
        uint64_t V = draw64(rule, Lx, Ly, xw, yw, zw, seed, s, a, t, u, d);
        d++;
        int rem = n - start;
        if (V >= C[rem])
            break; /* no selection among the remaining sites */
        int G = 0;
        while (!(V < C[G + 1]))
            G++;
        selected |= 1u << list[start + G];
        start += G + 1;
    }
    return selected;
}

/* What one temperature and rule fix for every word-site: always[k] (k =
   (dE + 12) / 4) marks the Metropolis classes accepted outright; live[u] the
   classes u = 0, 1, 2 decided by the gap table C[u] (for the heat bath, table
   u also serves class 6 - u). */
struct flip_rule {
    int rule;
    uint8_t always[7];
    int live[3];
    uint64_t C[3][33];
};

static int flip_rule_init(double T, int rule, struct flip_rule *f)
{
    uint64_t thr[7];
    if (ora_thresholds(T, rule, thr, f->always) != ORA_OK)
        return ORA_BAD_ARG;
    f->rule = rule;
    for (int u = 0; u < 3; u++) {
        double p;
        f->live[u] = 0;
        if (rule == 0) {
            int k = 6 - u;
            if (f->always[k] || thr[k] == 0)
                continue;
            p = exp(-(double)(12 - 4 * u) / T);
        } else {
            if (T == 0.0)
                continue;
            p = 1.0 / (1.0 + exp((double)(12 - 4 * u) / T));
            if (!(p > 0.0))
                continue;
        }
        f->live[u] = 1;
        ora_geo_table(p, f->C[u]);
    }
    return ORA_OK;
}

/* The lanes of class u (the mask `lanes`) of one word-site that flip:
     rule 0 (Metropolis): a class accepted outright (dE <= 0, or e^(-dE/T)
       rounding to 1) flips whole; a class with a gap table flips the lanes
       the gaps select; a class with threshold 0 never flips.
     rule 1 (heat bath), P(dE) = 1/(1+e^(dE/T)) and P(dE) + P(-dE) = 1:
       u = 0, 1, 2: the lanes the gaps of table u select flip;
       u = 3 (dE = 0, P = 1/2): lane b flips when bit b of the coin word is 1;
       u = 4, 5, 6: a lane keeps its spin with probability 1 - P(dE) =
         P(-dE), so the gaps of table 6 - u select the lanes that keep, and
         every other lane of the class flips.
       A table that is not live (p = 0: T = 0 or e^(dE/T) beyond the double
       range) leaves class u < 3 unflipped and flips all of class 6 - u. */
static uint32_t class_flips(const struct flip_rule *f, uint32_t lanes, int Lx, int Ly, int xw,
                            int yw, int zw, uint64_t seed, uint32_t s, int a, uint64_t t, int u)
{
    if (lanes == 0)
        return 0;
    if (f->rule == 0) {
        if (f->always[6 - u])
            return lanes;
        if (u >= 3 || !f->live[u])
            return 0;
        return gap_select(f->C[u], lanes, 0, Lx, Ly, xw, yw, zw, seed, s, a, t, u);
    }
    if (u == 3) {
        uint32_t coin = coin_word(Lx, Ly, xw, yw, zw, seed, s, a, t);
        return lanes & coin;
    }
    int j = u < 3 ? u : 6 - u;
    uint32_t mark = f->live[j] ? gap_select(f->C[j], lanes, 1, Lx, Ly, xw, yw, zw, seed, s, a,
                                            t, u)
                               : 0;
    return u < 3 ? mark : (lanes & ~mark);
}

/* Word-site arguments of the exported draw functions. */
static int word_site_ok(int L, int xw, int yw, int zw, int g[6])
{
    if (ora_geometry(L, g) != ORA_OK)
        return 0;
    return xw >= 0 && yw >= 0 && zw >= 0 && xw < g[3] && yw < g[4] && zw < g[5];
}

/* Draw d of class u (for the pins of the draw contract). */
int ora_draw64(int rule, int L, uint64_t seed, uint32_t s, int a, uint64_t t, int xw, int yw,
               int zw, int u, int d, uint64_t *out)
{
    int g[6];
    int u_ok = rule == 0 ? (u >= 0 && u <= 2) : (rule == 1 && u >= 0 && u <= 6 && u != 3);
    if (!word_site_ok(L, xw, yw, zw, g) || !u_ok || d < 0 || d > 31 || (a != 0 && a != 1) ||
        t >= ((uint64_t)1 << 48))
        return ORA_BAD_ARG;
    *out = draw64(rule, g[3], g[4], xw, yw, zw, seed, s, a, t, u, d);
    return ORA_OK;
}

/* The heat bath's coin word (for the pins). */
int ora_coin_word(int L, uint64_t seed, uint32_t s, int a, uint64_t t, int xw, int yw, int zw,
                  uint32_t *out)
{
    int g[6];
    if (!word_site_ok(L, xw, yw, zw, g) || (a != 0 && a != 1) || t >= ((uint64_t)1 << 48))
        return ORA_BAD_ARG;
    *out = coin_word(g[3], g[4], xw, yw, zw, seed, s, a, t);
    return ORA_OK;
}

/* The flips of class u among the lanes `lanes` of word-site (xw, yw, zw) at
   the sweeps t0, t0 + 1, ..., t0 + n_t - 1 (out[k] for sweep t0 + k): the
   decision the half-step takes for that class (for the pins). */
int ora_class_flips(int rule, int L, double T, uint64_t seed, uint32_t s, int a, uint64_t t0,
                    int n_t, int xw, int yw, int zw, int u, uint32_t lanes, uint32_t *out)
{
    int g[6];
    struct flip_rule f;
    if (!word_site_ok(L, xw, yw, zw, g) || u < 0 || u > 6 || (a != 0 && a != 1) || n_t < 0 ||
        t0 + (uint64_t)n_t > ((uint64_t)1 << 48) || (rule != 0 && rule != 1) ||
        flip_rule_init(T, rule, &f) != ORA_OK)
        return ORA_BAD_ARG;
    int lanes_max = g[0] * g[1] * g[2];
    if (lanes_max < 32 && (lanes >> lanes_max) != 0)
        return ORA_BAD_ARG;
    for (int k = 0; k < n_t; k++)
        out[k] = class_flips(&f, lanes, g[3], g[4], xw, yw, zw, seed, s, a, t0 + (uint64_t)k, u);
    return ORA_OK;
}

/* Local field dE = 2 S_i sum_j J_ij S_j at site (x, y, z) of replica Sa. */
static int delta_E(int L, const int8_t *Sa, const int8_t *J, int x, int y, int z)
{
    int64_t N = (int64_t)L * L * L;
    int64_t i = x + (int64_t)L * (y + (int64_t)L * z);
    int xp = (x + 1) % L, xm = (x + L - 1) % L;
    int yp = (y + 1) % L, ym = (y + L - 1) % L;
    int zp = (z + 1) % L, zm = (z + L - 1) % L;
    int64_t ixp = xp + (int64_t)L * (y + (int64_t)L * z);
    int64_t ixm = xm + (int64_t)L * (y + (int64_t)L * z);
    int64_t iyp = x + (int64_t)L * (yp + (int64_t)L * z);
    int64_t iym = x + (int64_t)L * (ym + (int64_t)L * z);
    int64_t izp = x + (int64_t)L * (y + (int64_t)L * zp);
    int64_t izm = x + (int64_t)L * (y + (int64_t)L * zm);
    /* forward bonds are stored at i, backward bonds at the neighbour i - e_d */
    int h_loc = J[0 * N + i] * Sa[ixp] + J[0 * N + ixm] * Sa[ixm] + J[1 * N + i] * Sa[iyp] +
                J[1 * N + iym] * Sa[iym] + J[2 * N + i] * Sa[izp] + J[2 * N + izm] * Sa[izm];
    return 2 * Sa[i] * h_loc;
}

/* ------------------------------------------------------------------------ */
/* Half-step h of sweep t of both replicas of one sample (Sec. III): replica */
/* a updates every site of colour (x+y+z) mod 2 equal to h XOR a.  Sites of  */
/* one colour do not neighbour each other, so the sites of a colour are     */
/* decided from the same configuration and may be taken in any order; here  */
/* they are taken word-site by word-site.  Each site gets dE = 2 S_i sum_j  */
/* J_ij S_j (Eq. 9) and class u = (12 - dE) / 4, and each class of the      */
/* word-site flips as class_flips decides.  dE_acc[a] accumulates the       */
/* energy change of accepted flips of replica a.  s keys the random numbers */
/* (counter word 3): the sample index, or the sample index divided by G     */
/* when G samples share their random numbers.                               */
/* ------------------------------------------------------------------------ */
int ora_half_step(int L, uint64_t seed, uint32_t s, int8_t *S, const int8_t *J, double T, int rule,
                  uint64_t t, int h, int64_t dE_acc[2])
{
    struct flip_rule f;
    if (L < 2 || L > 1024 || (L & 1) || t >= ((uint64_t)1 << 48) || (h != 0 && h != 1) ||
        (rule != 0 && rule != 1) || flip_rule_init(T, rule, &f) != ORA_OK)
        return ORA_BAD_ARG;
    int g[6];
    ora_geometry(L, g);
    int kx = g[0], ky = g[1], kz = g[2], Lx = g[3], Ly = g[4], Lz = g[5];
    int lanes = kx * ky * kz;
    int64_t N = (int64_t)L * L * L;
    for (int a = 0; a < 2; a++) {
        int8_t *Sa = S + a * N;
        for (int zw = 0; zw < Lz; zw++)
            for (int yw = 0; yw < Ly; yw++)
                for (int xw = 0; xw < Lx; xw++) {
                    if (((xw + yw + zw) & 1) != (h ^ a))
                        continue;
                    int dE[32], sx[32], sy[32], sz[32];
                    uint32_t in_class[7] = {0, 0, 0, 0, 0, 0, 0};
                    for (int b = 0; b < lanes; b++) {
                        sx[b] = (b % kx) * Lx + xw;
                        sy[b] = ((b / kx) % ky) * Ly + yw;
                        sz[b] = (b / (kx * ky)) * Lz + zw;
                        dE[b] = delta_E(L, Sa, J, sx[b], sy[b], sz[b]);
                        in_class[(12 - dE[b]) / 4] |= 1u << b;
                    }
                    uint32_t flips = 0;
                    for (int u = 0; u <= 6; u++)
                        flips |= class_flips(&f, in_class[u], Lx, Ly, xw, yw, zw, seed, s, a, t,
                                             u);
                    for (int b = 0; b < lanes; b++)
                        if ((flips >> b) & 1u) {
                            int64_t i = sx[b] + (int64_t)L * (sy[b] + (int64_t)L * sz[b]);
                            Sa[i] = (int8_t)-Sa[i];
                            dE_acc[a] += dE[b];
                        }
                }
    }
    return ORA_OK;
}

/* One sweep t: half-step 0, then half-step 1. */
int ora_sweep(int L, uint64_t seed, uint32_t s, int8_t *S, const int8_t *J, double T, int rule,
              uint64_t t, int64_t dE_acc[2])
{
    for (int h = 0; h < 2; h++) {
        int rc = ora_half_step(L, seed, s, S, J, T, rule, t, h, dE_acc);
        if (rc != ORA_OK)
            return rc;
    }
    return ORA_OK;
}

/* Several sweeps t0, t0+1, ..., t0+n-1 in a row. */
int ora_sweeps(int L, uint64_t seed, uint32_t s, int8_t *S, const int8_t *J, double T, int rule,
               uint64_t t0, uint64_t n, int64_t dE_acc[2])
{
    for (uint64_t k = 0; k < n; k++) {
        int rc = ora_sweep(L, seed, s, S, J, T, rule, t0 + k, dE_acc);
        if (rc != ORA_OK)
            return rc;
    }
    return ORA_OK;
}
