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
 * publication.  The mapping from (seed, sample, replica, site, sweep) to the
 * 64-bit uniform number compared against a threshold is a definition of this
 * library (the paper's generator cannot be reproduced); it is restated in
 * full in ora_random64 below.
 */
#include <math.h>
#include <stdint.h>
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
#define STREAM_SWEEP 2u

/* ------------------------------------------------------------------------ */
/* Lattice geometry of the random-number mapping.                           */
/*                                                                          */
/* A "word-site" groups up to 32 lattice sites of one sample that are drawn */
/* from the same Philox outputs, one bit each (see ora_random64).  The      */
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
/* The 64-bit uniform number r(seed, s, a, site, t) used by the heat-bath    */
/* update of replica a of sample s at the given site during sweep t.        */
/*                                                                          */
/* Bit (63 - k) of r, k = 0..63, is bit `lane` of plane k, where plane k is */
/* output word (k mod 4) of Philox4x32-10 with key (lo32(seed), hi32(seed)) */
/* and counter                                                              */
/*   c0 = widx, c1 = lo32(t),                                               */
/*   c2 = (2 << 30) | (bits 32..47 of t) << 8 | a << 4 | (k div 4),         */
/*   c3 = s.                                                                */
/* ------------------------------------------------------------------------ */
/* Bits 63..32 (half = 0, calls 0..7) or bits 31..0 (half = 1, calls 8..15)
   of r, as a 32-bit number. */
static uint32_t random_half(int L, uint64_t seed, uint32_t s, int a, int x, int y, int z, uint64_t t,
                            int half)
{
    uint32_t widx;
    int lane;
    site_to_word(L, x, y, z, &widx, &lane);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t v = 0;
    for (int call = 8 * half; call < 8 * half + 8; call++) {
        uint32_t ctr[4] = {widx, (uint32_t)t,
                           (STREAM_SWEEP << 30) | ((uint32_t)((t >> 32) & 0xFFFFu) << 8) |
                               ((uint32_t)a << 4) | (uint32_t)call,
                           s};
        uint32_t out[4];
        ora_philox4x32_10(ctr, key, out);
        for (int j = 0; j < 4; j++) {
            int k = 4 * call + j;          /* plane index, 0..63 */
            uint32_t bit = (out[j] >> lane) & 1u;
            v |= bit << (31 - (k - 32 * half));
        }
    }
    return v;
}

uint64_t ora_random64(int L, uint64_t seed, uint32_t s, int a, int x, int y, int z, uint64_t t)
{
    uint64_t hi = random_half(L, seed, s, a, x, y, z, t, 0);
    uint64_t lo = random_half(L, seed, s, a, x, y, z, t, 1);
    return (hi << 32) | lo;
}

/* r < thr for r = ora_random64(...).  Two 64-bit numbers compare by their
   top 32 bits unless those are equal, so the bottom half is drawn only then. */
static int random_below(int L, uint64_t seed, uint32_t s, int a, int x, int y, int z, uint64_t t,
                        uint64_t thr)
{
    uint32_t r_hi = random_half(L, seed, s, a, x, y, z, t, 0);
    uint32_t t_hi = (uint32_t)(thr >> 32);
    if (r_hi != t_hi)
        return r_hi < t_hi;
    uint32_t r_lo = random_half(L, seed, s, a, x, y, z, t, 1);
    return r_lo < (uint32_t)thr;
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds, one per energy change dE = 4k - 12, k = 0..6.     */
/* A move with energy change dE is accepted when always[k] is set, or when  */
/* r < thr[k] for the 64-bit uniform r above, i.e. with probability         */
/* thr[k] / 2^64 = floor(2^64 P(dE)) / 2^64.                                */
/*   rule 0, Metropolis (Eq. 9):  P = min(1, exp(-dE/T))                    */
/*   rule 1, heat bath:           P = 1 / (1 + exp(dE/T))                   */
/* P == 1 sets always[k].  T = 0 and T = +inf are the limits of P.          */
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
/* Metropolis acceptance by geometric gaps.                                 */
/*                                                                          */
/* Among the sites of one word-site that share the energy change dE > 0     */
/* (class u = (12 - dE) / 4 unsatisfied bonds, u = 0, 1, 2), each must flip  */
/* independently with probability p_u = exp(-dE/T) (Eq. 9).  Taken in       */
/* increasing lane order, they form a Bernoulli(p_u) sequence, and the      */
/* number G of rejections before the first acceptance is geometric:         */
/* P(G >= g) = (1 - p_u)^g.  One 64-bit uniform V decides the first         */
/* acceptance among n remaining sites: none if V >= C_u[n], else the site   */
/* of rank G = min{g : V < C_u[g+1]}, with                                  */
/*   C_u[g] = floor(2^64 (1 - (1 - p_u)^g)),  computed as                   */
/*   floor(ldexp(-expm1(g * log1p(-p_u)), 64)), clamped to 2^64 - 1.         */
/* The sites after an acceptance start a fresh gap with the next draw.      */
/*                                                                          */
/* Draws.  Word-sites group in quads (x' even, x' + 1) x (z' even, z' + 1) */
/* of the word lattice: one Philox call per quad holds the leading bits of  */
/* the first draws of all four words:                                       */
/*   main call of the quad: counter (widx of its word (x' even, z' even),   */
/*     lo32(t), (3 << 30) | (bits 32..47 of t) << 12 | a_q << 11 | 0, s),     */
/*     where a_q is the replica updated at that word in this half-step;     */
/*     output k = (x' mod 2) + 2 (z' mod 2) belongs to word (x', y', z'):    */
/*     its bits 31..20 are bits 63..52 of draw 0 of class 2 (dE = 4), bits  */
/*     19..10 bits 63..54 of class 1's (dE = 8), bits 9..0 bits 63..54 of   */
/*     class 0's (dE = 12).                                                 */
/*   extension calls of a word: counter (its widx, lo32(t), ... | a << 11 | */
/*     call, s).  Call 64: (out0 << 32 | out1) >> 12 = bits 51..0 of class */
/*     2's draw 0, (out2 << 32 | out3) >> 10 = bits 53..0 of class 1's.    */
/*     Call 65: (out0 << 32 | out1) >> 10 = bits 53..0 of class 0's.        */
/*   draw d >= 1 of class u of a word: the 64-bit number (out[2e] << 32) |   */
/*     out[2e + 1] of call 1 + u + 3 (d-1 div 2), e = (d-1) mod 2, with the   */
/*     word's own widx and replica.                                          */
#define STREAM_METROPOLIS 3u

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

static void metro_call(uint32_t widx, uint64_t seed, uint32_t s, int a, uint64_t t, int call,
                       uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {widx, (uint32_t)t,
                       (STREAM_METROPOLIS << 30) | ((uint32_t)((t >> 32) & 0xFFFFu) << 12) |
                           ((uint32_t)a << 11) | (uint32_t)call,
                       s};
    ora_philox4x32_10(ctr, key, out);
}

/* Draw d of class u for the word-site (xw, yw, zw) of a lattice whose word
   lattice is Lx x Ly x Lz, updated in replica a. */
static uint64_t metro_draw(int Lx, int Ly, int xw, int yw, int zw, uint64_t seed, uint32_t s,
                           int a, uint64_t t, int u, int d)
{
    uint32_t widx = (uint32_t)(xw + Lx * (yw + Ly * zw));
    if (d >= 1) {
        uint32_t out[4];
        int e = (d - 1) % 2;
        metro_call(widx, seed, s, a, t, 1 + u + 3 * ((d - 1) / 2), out);
        return ((uint64_t)out[2 * e] << 32) | (uint64_t)out[2 * e + 1];
    }
    /* leading bits from the quad's main call */
    int ox = xw & 1, oz = zw & 1;
    uint32_t widx_q = (uint32_t)((xw - ox) + Lx * (yw + Ly * (zw - oz)));
    int a_q = a ^ ox ^ oz; /* the replica updated at the quad's first word */
    uint32_t m[4], x[4];
    metro_call(widx_q, seed, s, a_q, t, 0, m);
    uint32_t lead = m[ox + 2 * oz];
    if (u == 2) {
        metro_call(widx, seed, s, a, t, 64, x);
        return ((uint64_t)(lead >> 20) << 52) | ((((uint64_t)x[0] << 32) | x[1]) >> 12);
    }
    if (u == 1) {
        metro_call(widx, seed, s, a, t, 64, x);
        return ((uint64_t)((lead >> 10) & 0x3FFu) << 54) | ((((uint64_t)x[2] << 32) | x[3]) >> 10);
    }
    metro_call(widx, seed, s, a, t, 65, x);
    return ((uint64_t)(lead & 0x3FFu) << 54) | ((((uint64_t)x[0] << 32) | x[1]) >> 10);
}

/* Flip decisions of the lanes lane_list[0..n) (increasing lane order) of one
   class: sets flip[lane] = 1 for the accepted ones. */
static void metro_class(const uint64_t C[33], const int *lane_list, int n, int Lx, int Ly,
                        int xw, int yw, int zw, uint64_t seed, uint32_t s, int a, uint64_t t,
                        int u, uint8_t *flip)
{
    int start = 0, d = 0;
    while (n - start > 0) {
        uint64_t V = metro_draw(Lx, Ly, xw, yw, zw, seed, s, a, t, u, d);
        d++;
        int rem = n - start;
        if (V >= C[rem])
            break; /* no acceptance among the remaining sites */
        int G = 0;
        while (!(V < C[G + 1]))
            G++;
        flip[lane_list[start + G]] = 1;
        start += G + 1;
    }
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
/* J_ij S_j (Eq. 9), k = (dE + 12) / 4, and flips when always[k];           */
/*   rule 0 (Metropolis): the other sites of a word-site are decided per    */
/*     class by geometric gaps (above); a class with threshold 0 never flips */
/*   rule 1 (heat bath): a site flips when its uniform r < thr[k]           */
/*     (ora_random64).                                                      */
/* dE_acc[a] accumulates the energy change of accepted flips of replica a.  */
/* s keys the random numbers (counter word 3): the sample index, or the     */
/* sample index divided by G when G samples share their random numbers.     */
/* ------------------------------------------------------------------------ */
int ora_half_step(int L, uint64_t seed, uint32_t s, int8_t *S, const int8_t *J, double T, int rule,
                  uint64_t t, int h, int64_t dE_acc[2])
{
    uint64_t thr[7];
    uint8_t always[7];
    if (L < 2 || L > 1024 || (L & 1) || t >= ((uint64_t)1 << 48) || (h != 0 && h != 1) ||
        ora_thresholds(T, rule, thr, always) != ORA_OK)
        return ORA_BAD_ARG;
    uint64_t C[3][33];
    int live[3] = {0, 0, 0};
    if (rule == 0) {
        for (int u = 0; u < 3; u++) {
            int k = 6 - u;
            if (!always[k] && thr[k] > 0) {
                live[u] = 1;
                ora_geo_table(exp(-(double)(12 - 4 * u) / T), C[u]);
            }
        }
    }
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
                    uint8_t flip[32];
                    for (int b = 0; b < lanes; b++) {
                        sx[b] = (b % kx) * Lx + xw;
                        sy[b] = ((b / kx) % ky) * Ly + yw;
                        sz[b] = (b / (kx * ky)) * Lz + zw;
                        dE[b] = delta_E(L, Sa, J, sx[b], sy[b], sz[b]);
                        flip[b] = always[(dE[b] + 12) / 4];
                    }
                    if (rule == 0) {
                        for (int u = 0; u < 3; u++) {
                            if (!live[u])
                                continue;
                            int list[32], n = 0;
                            for (int b = 0; b < lanes; b++)
                                if (dE[b] == 12 - 4 * u)
                                    list[n++] = b;
                            if (n > 0)
                                metro_class(C[u], list, n, Lx, Ly, xw, yw, zw, seed, s, a, t,
                                            u, flip);
                        }
                    } else {
                        for (int b = 0; b < lanes; b++)
                            if (!flip[b])
                                flip[b] = (uint8_t)random_below(L, seed, s, a, sx[b], sy[b],
                                                                sz[b], t, thr[(dE[b] + 12) / 4]);
                    }
                    for (int b = 0; b < lanes; b++)
                        if (flip[b]) {
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
