// ea_sweep.cu -- the checkerboard half-step kernels (Sec. III) over a table of jobs.
//
// In half-step h every word-site of area h is updated (it holds the replica
// whose colour is due in half-step h, Fig. 1); its neighbours are read from
// area 1 - h.  The kernels differ in how threads share that work:
//   metro_kernel, heat_kernel      a column of word-sites along z per thread,
//                                  any side, z-neighbours in a register window;
//   metro_tile_kernel,             2 x 2 word tiles over a segment of rows per
//   heat_tile_kernel               thread, sides 64 and 128 (all lanes along z);
//   metro_gtile_kernel             the same tiles for the other sides divisible
//                                  by 16 (lanes along y and z).
//
// Per word (32 sites of one sample):
//   u_j = s ^ n_j ^ J_j for the six bonds (1 = unsatisfied)         6 LOP3
//   bit-sliced count (b2 b1 b0) = u                                 8 LOP3
//   dE = 12 - 4u (Eq. 9).
//   Metropolis: u >= 3 (dE <= 0) flips outright.  The lanes of class u = 0, 1,
//     2 (dE = 12, 8, 4) flip independently with p_u = exp(-dE/T); taken in lane
//     order they form a Bernoulli sequence whose first acceptance rank is
//     geometric, so one 64-bit draw V per class decides: no flip when
//     V >= C_u[n] (n lanes in the class), else the lane of rank
//     min{g : V < C_u[g+1]}, after which the remaining lanes take the next
//     draw.  One Philox call per 2 x 2 quad of words holds the leading 12
//     (class 2) and 10 (classes 1, 0) bits of their first draws, enough to
//     settle ~97% of words at T = 0.7 without a branch; the rest of a draw is
//     fetched only when the test hits.
//   Heat bath: one Philox call per word holds a coin word for dE = 0 and the
//     leading bits of the first gap draws of the other six classes; classes
//     dE > 0 flip the lanes the gaps select, classes dE < 0 keep them
//     (P(dE) + P(-dE) = 1).
// Words whose leading bits might select a lane wait in a per-warp queue and
// are finished 32 at a time (the rare path), so it runs converged.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ea_device.cuh"
#include "ea_internal.h"

namespace ea {
namespace {

using dev::maj3;
using dev::realign;

struct Axis {
    int sA[2], sB[2];
    uint32_t mA[2], mB[2];
};

__device__ __forceinline__ uint32_t fixup(uint32_t w, const Axis &a, int dir)
{
    return realign(w, a.sA[dir], a.mA[dir], a.sB[dir], a.mB[dir]);
}

__device__ __forceinline__ void load_axis(Axis &a, const Geo &g, int d)
{
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        a.sA[dir] = g.sA[d][dir];
        a.sB[dir] = g.sB[d][dir];
        a.mA[dir] = g.mA[d][dir];
        a.mB[dir] = g.mB[d][dir];
    }
}

// The bit-sliced count u = 4 b2 + 2 b1 + b0 of six unsatisfied-bond bits.
struct Count {
    uint32_t b0, b1, b2;
};

__device__ __forceinline__ Count count6(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3,
                                        uint32_t u4, uint32_t u5)
{
    const uint32_t s1 = u0 ^ u1 ^ u2, k1 = maj3(u0, u1, u2);
    const uint32_t s2 = u3 ^ u4 ^ u5, k2 = maj3(u3, u4, u5);
    Count c;
    c.b0 = s1 ^ s2;
    const uint32_t k3 = s1 & s2;
    c.b1 = k1 ^ k2 ^ k3;
    c.b2 = maj3(k1, k2, k3);
    return c;
}

// ---------------------------------------------------------------------------
// Metropolis draws.  Word-sites group in quads (x' even, x' + 1) x (z' even,
// z' + 1); one Philox call per quad ("main", call 0, keyed by the quad's word
// (x' even, z' even) and its replica) holds the leading bits of the first
// draws of all four words.  Output k = (x' & 1) + 2 (z' & 1) belongs to word
// (x', y', z'): bits 31..20 lead class 2's draw 0 (bits 63..52), bits 19..10
// class 1's (63..54), bits 9..0 class 0's.  A word's extension calls (its
// own widx and replica) hold the rest: call 64 gives (out0:out1) >> 12 =
// bits 51..0 of class 2's draw and (out2:out3) >> 10 = bits 53..0 of class
// 1's; call 65 gives (out0:out1) >> 10 = bits 53..0 of class 0's.  Draw
// d >= 1 of class u is (out[2e] << 32) | out[2e + 1] of call
// 1 + u + 3 ((d - 1) div 2), e = (d - 1) mod 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t c64(const JobDev *__restrict__ jb, int u, int g)
{
    return ((uint64_t)jb->gC_hi[u][g] << 32) | jb->gC_lo[u][g];
}

// The lane (as a one-bit mask) of rank k among the set bits of m, k < popc(m).
__device__ __forceinline__ uint32_t nth_bit(uint32_t m, int k)
{
    int p = 0, c = __popc(m & 0xFFFFu);
    if (k >= c) {
        k -= c;
        p = 16;
    }
    c = __popc((m >> p) & 0xFFu);
    if (k >= c) {
        k -= c;
        p += 8;
    }
    c = __popc((m >> p) & 0xFu);
    if (k >= c) {
        k -= c;
        p += 4;
    }
    c = __popc((m >> p) & 0x3u);
    if (k >= c) {
        k -= c;
        p += 2;
    }
    if (k >= (int)((m >> p) & 1u))
        p += 1;
    return 1u << p;
}

// The lanes of Mr that the geometric gaps of table C_tab select, from the full
// first draw V0; draw d >= 1 is taken from call 1 + cu + STRIDE ((d - 1) div 2)
// (Metropolis: STRIDE 3 and cu = tab; heat bath: STRIDE 7, cu the class).
template <int STRIDE>
__device__ __forceinline__ uint32_t gap_class(const JobDev *__restrict__ jb, int tab, int cu,
                                              uint32_t Mr, uint64_t V0, uint32_t w, uint32_t c1,
                                              uint32_t c2, uint32_t c3, const uint32_t (&rk)[20],
                                              unsigned int &calls)
{
    uint32_t acc = 0u;
    int rem = __popc(Mr);
    int d = 0;
    uint64_t V = V0;
    while (rem > 0) {
        if (!(V < c64(jb, tab, rem)))
            break;  // no selection among the remaining lanes
        // G = min{g : V < C[g + 1]} by bisection over the nondecreasing table
        int lo = 1, hi = rem;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (V < c64(jb, tab, mid))
                hi = mid;
            else
                lo = mid + 1;
        }
        const int G = lo - 1;
        const uint32_t bit = nth_bit(Mr, G);  // the lane of rank G among the remaining ones
        acc |= bit;
        Mr &= ~(bit | (bit - 1u));
        rem -= G + 1;
        if (rem == 0)
            break;
        ++d;
        const int e = (d - 1) & 1;
        const uint4 Q = dev::philox10_rk(
            make_uint4(w, c1, c2 | (uint32_t)(1 + cu + STRIDE * ((d - 1) >> 1)), c3), rk);
        ++calls;
        V = e == 0 ? (((uint64_t)Q.x << 32) | Q.y) : (((uint64_t)Q.z << 32) | Q.w);
    }
    return acc;
}

// The accepted lanes of Metropolis class u of a word, from its full first draw V0.
__device__ __forceinline__ uint32_t metro_class(const JobDev *__restrict__ jb, int u, uint32_t Mr,
                                                uint64_t V0, uint32_t w, uint32_t c1,
                                                uint32_t c2, uint32_t c3, const uint32_t (&rk)[20],
                                                unsigned int &calls)
{
    return gap_class<3>(jb, u, u, Mr, V0, w, c1, c2, c3, rk, calls);
}

// Class masks of a word (u = 0, 1, 2 <=> b2 = 0 and not b1 & b0)
struct Classes {
    uint32_t M0, M1, M2;
};

__device__ __forceinline__ Classes classes(const Count &c, uint32_t alw, uint32_t valid,
                                           uint32_t live0, uint32_t live1, uint32_t live2)
{
    const uint32_t need = ~alw & valid;
    Classes k;
    k.M0 = need & ~(c.b1 | c.b0) & live0;
    k.M1 = need & c.b0 & live1;
    k.M2 = need & c.b1 & live2;
    return k;
}

// Leading-bit tables: a word's 32 main bits M might accept a lane of class 2
// iff M <= lead2(C_2[n]), of class 1 iff (M & 0xFFC00) <= lead1(C_1[n]), of
// class 0 iff (M & 0x3FF) <= lead0(C_0[n]); hi = C_u[n] >> 32.
__device__ __forceinline__ uint32_t lead2(uint32_t hi)
{
    return (hi & 0xFFF00000u) | 0xFFFFFu;
}

__device__ __forceinline__ uint32_t lead1(uint32_t hi)
{
    return ((hi >> 22) << 10) | 0x3FFu;
}

__device__ __forceinline__ uint32_t lead0(uint32_t hi)
{
    return hi >> 22;
}

// Might some lane of the word flip?  The leading bits of the first draws
// against the tables (lead2, lead1, lead0 of C_u[n]): an exact "no" for ~97%
// of words at T = 0.7.
__device__ __forceinline__ bool class_hit(const Classes &k, uint32_t M, const uint32_t (*gh)[33])
{
    const int n0 = __popc(k.M0), n1 = __popc(k.M1), n2 = __popc(k.M2);
    const bool h2 = (n2 != 0) & (M <= gh[2][n2]);
    const bool h1 = (n1 != 0) & ((M & 0xFFC00u) <= gh[1][n1]);
    const bool h0 = (n0 != 0) & ((M & 0x3FFu) <= gh[0][n0]);
    return h0 | h1 | h2;
}

// The first draw of class u of a word from its main bits M and its extension
// calls X (call 64) and Y (call 65).
__device__ __forceinline__ uint64_t first_draw2(uint32_t M, const uint4 &X)
{
    return ((uint64_t)(M >> 20) << 52) | ((((uint64_t)X.x << 32) | X.y) >> 12);
}

__device__ __forceinline__ uint64_t first_draw1(uint32_t M, const uint4 &X)
{
    return ((uint64_t)((M >> 10) & 0x3FFu) << 54) | ((((uint64_t)X.z << 32) | X.w) >> 10);
}

__device__ __forceinline__ uint64_t first_draw0(uint32_t M, const uint4 &Y)
{
    return ((uint64_t)(M & 0x3FFu) << 54) | ((((uint64_t)Y.x << 32) | Y.y) >> 10);
}

// Words whose class test hit wait in a per-warp queue and are finished by the
// whole warp at once, one word per lane, so the rare path runs converged.
constexpr int kQueue = 96;  // entries per warp (up to 64 are added per step)

struct Pending {
    uint32_t w, base, M0, M1, M2, c2, lead;  // lead: the word's 32 main bits
};

__device__ __forceinline__ void finish_word(const JobDev *__restrict__ jb, const Pending &e,
                                            uint32_t *__restrict__ upd, uint32_t valid,
                                            uint32_t c1, uint32_t c3, const uint32_t (&rk)[20],
                                            unsigned int &calls)
{
    // the extension call completes the first draws of classes 2 and 1
    const uint4 X = dev::philox10_rk(make_uint4(e.w, c1, e.c2 | 64u, c3), rk);
    ++calls;
    uint32_t A = 0u, M0 = e.M0, M1 = e.M1, M2 = e.M2;
    const uint32_t always3 = jb->always_u & 7u;
    if (always3) {  // classes accepted outright (exp(-dE/T) rounds to 1)
        A = ((always3 & 4u) ? M2 : 0u) | ((always3 & 2u) ? M1 : 0u) | ((always3 & 1u) ? M0 : 0u);
        M2 = (always3 & 4u) ? 0u : M2;
        M1 = (always3 & 2u) ? 0u : M1;
        M0 = (always3 & 1u) ? 0u : M0;
    }
    if (M2)
        A |= metro_class(jb, 2, M2, first_draw2(e.lead, X), e.w, c1, e.c2, c3, rk, calls);
    if (M1)
        A |= metro_class(jb, 1, M1, first_draw1(e.lead, X), e.w, c1, e.c2, c3, rk, calls);
    // class 0 needs its own extension call, unless its leading bits rule it out
    if (M0 && (e.lead & 0x3FFu) <= lead0(jb->gC_hi[0][__popc(M0)])) {
        const uint4 Y = dev::philox10_rk(make_uint4(e.w, c1, e.c2 | 65u, c3), rk);
        ++calls;
        A |= metro_class(jb, 0, M0, first_draw0(e.lead, Y), e.w, c1, e.c2, c3, rk, calls);
    }
    upd[e.w] = e.base ^ (A & valid);
}

// Any side: the geometry is read from the job table.  A thread updates a
// column of word-sites along z.
template <bool COUNT, int MAXJ>
__global__ void __launch_bounds__(kSweepThreads, 10)
    metro_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    // the job of this block, found from blockIdx alone: the loads below stay
    // in the uniform datapath
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];  // round keys of the job's Philox key (block-uniform)
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    __shared__ uint32_t s_gh[3][33];
    __shared__ Pending s_q[kSweepThreads / 32][kQueue];
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33;
        const uint32_t hi = (&jb->gC_hi[0][0])[i];
        (&s_gh[0][0])[i] = u == 2 ? lead2(hi) : u == 1 ? lead1(hi) : lead0(hi);
    }
    __syncthreads();
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;  // this job has stopped (uniform over the block)

    const int h = P.h;
    const int lane = threadIdx.x & 31;
    Pending *q = s_q[threadIdx.x >> 5];
    int q_n = 0;  // warp-uniform queue length
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    const int cb = local - s * G.bps;
    const int n0 = G.n0, n1 = G.n1, n2 = G.n2;
    const bool all_always = (J.meta >> 3) & 1u, none_random = (J.meta >> 4) & 1u;
    const bool fix_x = (G.fix & 1u) != 0;
    const bool fix_y = (G.fix & 2u) != 0;
    const uint32_t valid = G.valid;
    const uint32_t live0 = 0u - (J.meta & 1u), live1 = 0u - ((J.meta >> 1) & 1u),
                   live2 = 0u - ((J.meta >> 2) & 1u);
    Axis az, ax, ay;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        az.sA[dir] = G.zsA[dir];
        az.sB[dir] = G.zsB[dir];
        az.mA[dir] = G.zmA[dir];
        az.mB[dir] = G.zmB[dir];
    }
    if (fix_x)
        load_axis(ax, jb->geo, 0);
    if (fix_y)
        load_axis(ay, jb->geo, 1);
    const uint32_t W = G.words;
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2m = dev::kStreamMetropolis | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    const int sz = n0 * n1;
    unsigned int n_words = 0, n_calls = 0, n_extra = 0;

    const int cols = G.cols;
    for (int k = 0; k < G.cpt; ++k) {
        const int col0 = (cb * G.cpt + k) * kSweepThreads + (int)threadIdx.x;
        // lanes past the last column idle in step
        const bool act = col0 < cols;
        if (__all_sync(0xffffffffu, !act))
            break;
        const int col = act ? col0 : 0;
        const int y = (int)((__umulhi((uint32_t)col, G.magic) + (uint32_t)col) >> G.dshift);
        const int x = col - y * n0;
        int cxp = col + 1, cxm = col - 1, cyp = col + n0, cym = col - n0;
        const bool wxp = (x + 1 == n0), wxm = (x == 0), wyp = (y + 1 == n1), wym = (y == 0);
        if (wxp)
            cxp = col - (n0 - 1);
        if (wxm)
            cxm = col + (n0 - 1);
        if (wyp)
            cyp = col - (n1 - 1) * n0;
        if (wym)
            cym = col + (n1 - 1) * n0;
        // replica updated at word-site (x, y, z) in half-step h: h ^ ((x + y + z) & 1)
        const uint32_t c2e = c2m | ((uint32_t)(h ^ ((x + y) & 1)) << 11);      // even z
        const uint32_t c2o = c2m | ((uint32_t)(h ^ ((x + y + 1) & 1)) << 11);  // odd z
        const int xo = x & 1;                                                   // odd x
        const uint32_t c2q = c2e ^ ((uint32_t)xo << 11);  // the quad's first word
        // z window: neighbour area at z' - 1 and the backward z bond below z'
        uint32_t nz_prev = fixup(nb[col + (n2 - 1) * sz], az, 1);
        uint32_t jz_prev = fixup(Jz[col + (n2 - 1) * sz], az, 1);
        uint32_t nz_cur = nb[col];
        for (int z = 0; z < n2; z += 2) {  // n2 is even: words at z (a) and z + 1 (b)
            const int wa = col + z * sz, wb = wa + sz;
            const uint32_t nz_b = nb[wb];                                             // z + 1
            const uint32_t nz_n = (z + 2 < n2) ? nb[wb + sz] : fixup(nb[col], az, 0);  // z + 2
            const uint32_t spa = upd[wa], spb = upd[wb];
            uint32_t nxpa = nb[cxp + z * sz], nxma = nb[cxm + z * sz];
            uint32_t nypa = nb[cyp + z * sz], nyma = nb[cym + z * sz];
            uint32_t jxma = Jx[cxm + z * sz], jyma = Jy[cym + z * sz];
            uint32_t nxpb = nb[cxp + z * sz + sz], nxmb = nb[cxm + z * sz + sz];
            uint32_t nypb = nb[cyp + z * sz + sz], nymb = nb[cym + z * sz + sz];
            uint32_t jxmb = Jx[cxm + z * sz + sz], jymb = Jy[cym + z * sz + sz];
            const uint32_t jxa = Jx[wa], jya = Jy[wa], jza = Jz[wa];
            const uint32_t jxb = Jx[wb], jyb = Jy[wb], jzb = Jz[wb];
            if (fix_x) {
                if (wxp) {
                    nxpa = fixup(nxpa, ax, 0);
                    nxpb = fixup(nxpb, ax, 0);
                }
                if (wxm) {
                    nxma = fixup(nxma, ax, 1);
                    nxmb = fixup(nxmb, ax, 1);
                    jxma = fixup(jxma, ax, 1);
                    jxmb = fixup(jxmb, ax, 1);
                }
            }
            if (fix_y) {
                if (wyp) {
                    nypa = fixup(nypa, ay, 0);
                    nypb = fixup(nypb, ay, 0);
                }
                if (wym) {
                    nyma = fixup(nyma, ay, 1);
                    nymb = fixup(nymb, ay, 1);
                    jyma = fixup(jyma, ay, 1);
                    jymb = fixup(jymb, ay, 1);
                }
            }
            // word b's -z neighbour is the neighbour area at z; its backward z bond is jza
            const Count ca = count6(spa ^ nxpa ^ jxa, spa ^ nxma ^ jxma, spa ^ nypa ^ jya,
                                    spa ^ nyma ^ jyma, spa ^ nz_b ^ jza, spa ^ nz_prev ^ jz_prev);
            const Count cw = count6(spb ^ nxpb ^ jxb, spb ^ nxmb ^ jxmb, spb ^ nypb ^ jyb,
                                    spb ^ nymb ^ jymb, spb ^ nz_n ^ jzb, spb ^ nz_cur ^ jza);
            nz_prev = nz_b;
            nz_cur = nz_n;
            jz_prev = jzb;

            const uint32_t alwa = ca.b2 | (ca.b1 & ca.b0);  // u >= 3 <=> dE <= 0
            const uint32_t alwb = cw.b2 | (cw.b1 & cw.b0);
            if (all_always || none_random) {
                if (act) {
                    upd[wa] = spa ^ ((all_always ? 0xffffffffu : alwa) & valid);
                    upd[wb] = spb ^ ((all_always ? 0xffffffffu : alwb) & valid);
                }
                if (COUNT && act)
                    n_words += 2;
                continue;
            }
            const Classes ka = classes(ca, alwa, valid, live0, live1, live2);
            const Classes kb = classes(cw, alwb, valid, live0, live1, live2);
            // leading bits of the first draws: the main call of the quad
            // (x & ~1, y, z | z + 1), computed by both of its columns
            const uint4 Rm = dev::philox10_rk(make_uint4((uint32_t)(wa - xo), c1, c2q, c3), rk);
            if (COUNT && act)
                n_calls += 1;
            const uint32_t La = xo ? Rm.y : Rm.x, Lb = xo ? Rm.w : Rm.z;
            const bool ha = act && class_hit(ka, La, s_gh);
            const bool hb = act && class_hit(kb, Lb, s_gh);
            const uint32_t basea = spa ^ (alwa & valid), baseb = spb ^ (alwb & valid);
            if (act && !ha)
                upd[wa] = basea;
            if (act && !hb)
                upd[wb] = baseb;
            if (COUNT && act)
                n_words += 2;
            // queue the words that may flip more lanes
            const uint32_t ba = __ballot_sync(0xffffffffu, ha);
            const uint32_t bbm = __ballot_sync(0xffffffffu, hb);
            const uint32_t below_me = (1u << lane) - 1u;
            if (ha) {
                Pending &e = q[q_n + __popc(ba & below_me)];
                e.w = (uint32_t)wa;
                e.base = basea;
                e.M0 = ka.M0;
                e.M1 = ka.M1;
                e.M2 = ka.M2;
                e.c2 = c2e;
                e.lead = La;
            }
            q_n += __popc(ba);
            if (hb) {
                Pending &e = q[q_n + __popc(bbm & below_me)];
                e.w = (uint32_t)wb;
                e.base = baseb;
                e.M0 = kb.M0;
                e.M1 = kb.M1;
                e.M2 = kb.M2;
                e.c2 = c2o;
                e.lead = Lb;
            }
            q_n += __popc(bbm);
            __syncwarp();
            while (q_n >= 32) {  // a full round: one queued word per lane
                q_n -= 32;
                const Pending e = q[q_n + lane];
                unsigned int extra = 0;
                finish_word(jb, e, upd, valid, c1, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
            }
        }
    }
    // the last, partial round
    if (lane < q_n) {
        const Pending e = q[lane];
        unsigned int extra = 0;
        finish_word(jb, e, upd, valid, c1, c3, rk, extra);
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_calls + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// ---------------------------------------------------------------------------
// Metropolis half-step for a table whose jobs all have side GL = 64 or 128.
// Their word lattice is GL x GL x GL/32 with all 32 lanes along z: x and y
// wrap without realignment, and a z wrap rotates the word by one lane.  A
// thread owns the word-sites (x0, x0 + 1) x (z0, z0 + 1), x0 and z0 even, of a
// segment of Y rows along y.  Rows y - 1 and y of the neighbour area and the y
// bonds of row y - 1 stay in registers from one row to the next, and the two
// words of an x pair are read and written as one 8-byte access.  The z pair
// is the pair that shares the main Philox call.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rot_zp(uint32_t w)  // +z neighbour across the wrap
{
    return __funnelshift_r(w, w, 1);
}

__device__ __forceinline__ uint32_t rot_zm(uint32_t w)  // -z neighbour across the wrap
{
    return __funnelshift_l(w, w, 1);
}

__device__ __forceinline__ uint2 ld2(const uint32_t *__restrict__ p, int i)
{
    return *reinterpret_cast<const uint2 *>(p + i);
}

constexpr int kGeneralTile = 1;  // run code of the general tile kernel (sides divisible by 16)
constexpr int kResidentRun = 2;  // run code of the sample-resident kernel
constexpr int kTileQueue = 224;  // entries per warp: up to 95 left over + 128 added per row
constexpr int kTileMinSMs = 152;  // SMs of a GB300: launches below 4 blocks per SM take shorter rows

// Threshold tables of a block's job in shared memory.
struct TileTables {
    uint32_t hi[3][33];    // C_u[n] >> 32
    uint32_t lead[3][33];  // lead0, lead1, lead2 of C_u[n]
};

// The rare path of one queued word: e = (word-site, spins before the update,
// its 32 main bits M, its class-2 lanes).  The row loop stored the word with
// its outright flips, which it reads back.  Class 2 is decided on the 12
// leading bits of its first draw and the full 64 bits of later draws; the
// extension call 64 is drawn only when those leading bits tie with the
// table.  Only when the 10 leading bits of class 1 or 0 fall at or below the
// class's 32-lane bound (T1x, T0) are the word's classes counted again from
// the neighbour area, which this half-step does not write, and decided
// exactly, with calls 64 and 65 as needed.
// The rare path of one queued word at word-site w with counter word c2, spins
// s, main bits M and class-2 lanes M2; `recount` counts the word's classes
// again from the neighbour area.
template <class Recount>
__device__ __forceinline__ void tile_finish_at(const JobDev *__restrict__ jb, const TileTables &tb,
                                               int w, uint32_t s, uint32_t M, uint32_t M2,
                                               uint32_t c2, uint32_t *__restrict__ upd,
                                               uint32_t live0, uint32_t live1, uint32_t live2,
                                               uint32_t always3, uint32_t T1x, uint32_t T0,
                                               uint32_t c1, uint32_t c3, const uint32_t (&rk)[20],
                                               unsigned int &calls, const Recount &recount)
{
    const uint32_t base = upd[w];  // s with its outright flips
    uint32_t A = 0u;
    if (always3 & 4u) {  // accepted outright (exp(-dE/T) rounds to 1)
        A = M2;
        M2 = 0u;
    }
    uint4 X = make_uint4(0u, 0u, 0u, 0u);
    bool have_x = false;
    if (M2) {
        uint32_t Mr = M2;
        int rem = __popc(Mr);
        uint32_t vh = M >> 20, vl = 0u;  // draw 0: its 12 leading bits until extended
        bool exact = false;
        int d = 0;
        // V < C_2[g]: by the leading bits unless they tie, then by all 64
        auto below = [&](int g) -> bool {
            const uint32_t ch = tb.hi[2][g];
            if (!exact) {
                const uint32_t c12 = ch >> 20;
                if (vh != c12)
                    return vh < c12;
                if (!have_x) {
                    X = dev::philox10_rk(make_uint4((uint32_t)w, c1, c2 | 64u, c3), rk);
                    ++calls;
                    have_x = true;
                }
                const uint64_t V = first_draw2(M, X);
                vh = (uint32_t)(V >> 32);
                vl = (uint32_t)V;
                exact = true;
            }
            if (vh != ch)
                return vh < ch;
            return vl < jb->gC_lo[2][g];
        };
        while (below(rem)) {
            // G = min{g : V < C_2[g + 1]} by bisection over the nondecreasing table
            int lo = 1, hi = rem;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (below(mid))
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int G = lo - 1;
            const uint32_t bit = nth_bit(Mr, G);  // the lane of rank G among the remaining ones
            A |= bit;
            Mr &= ~(bit | (bit - 1u));
            rem -= G + 1;
            if (rem == 0)
                break;
            ++d;
            const uint4 Q = dev::philox10_rk(
                make_uint4((uint32_t)w, c1, c2 | (uint32_t)(3 + 3 * ((d - 1) >> 1)), c3), rk);
            ++calls;
            const bool odd = ((d - 1) & 1) != 0;
            vh = odd ? Q.z : Q.x;
            vl = odd ? Q.w : Q.y;
            exact = true;
        }
    }
    if ((M & 0xFFC00u) <= T1x || (M & 0x3FFu) <= T0) {
        const Count c = recount();
        const uint32_t alw = c.b2 | (c.b1 & c.b0);
        const Classes k = classes(c, alw, 0xffffffffu, live0, live1, live2);
        uint32_t M1 = k.M1, M0 = k.M0;
        if (always3 & 2u) {
            A |= M1;
            M1 = 0u;
        }
        if (always3 & 1u) {
            A |= M0;
            M0 = 0u;
        }
        if (M1 && (M & 0xFFC00u) <= tb.lead[1][__popc(M1)]) {
            if (!have_x) {
                X = dev::philox10_rk(make_uint4((uint32_t)w, c1, c2 | 64u, c3), rk);
                ++calls;
            }
            A |= metro_class(jb, 1, M1, first_draw1(M, X), (uint32_t)w, c1, c2, c3, rk, calls);
        }
        if (M0 && (M & 0x3FFu) <= tb.lead[0][__popc(M0)]) {
            const uint4 Y = dev::philox10_rk(make_uint4((uint32_t)w, c1, c2 | 65u, c3), rk);
            ++calls;
            A |= metro_class(jb, 0, M0, first_draw0(M, Y), (uint32_t)w, c1, c2, c3, rk, calls);
        }
    }
    upd[w] = base ^ A;
}

template <int GL>
__device__ __forceinline__ void tile_finish(const JobDev *__restrict__ jb, const TileTables &tb,
                                            const uint4 &e, uint32_t *__restrict__ upd,
                                            const uint32_t *__restrict__ nb,
                                            const uint32_t *__restrict__ Jx,
                                            const uint32_t *__restrict__ Jy,
                                            const uint32_t *__restrict__ Jz, int h, uint32_t live0,
                                            uint32_t live1, uint32_t live2, uint32_t always3,
                                            uint32_t T1x, uint32_t T0, uint32_t c1, uint32_t c2m,
                                            uint32_t c3, const uint32_t (&rk)[20],
                                            unsigned int &calls)
{
    constexpr int SLOG = GL == 128 ? 7 : 6;
    constexpr int N2 = GL / 32, SZ = GL * GL;
    const int w = (int)e.x;
    const uint32_t s = e.y, M = e.z, M2 = e.w;
    const int x = w & (GL - 1), y = (w >> SLOG) & (GL - 1), z = w >> (2 * SLOG);
    const uint32_t c2 = c2m | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
    const auto recount = [&]() -> Count {
        const int wxp = x == GL - 1 ? w - (GL - 1) : w + 1;
        const int wxm = x == 0 ? w + (GL - 1) : w - 1;
        const int wyp = y == GL - 1 ? w - (GL - 1) * GL : w + GL;
        const int wym = y == 0 ? w + (GL - 1) * GL : w - GL;
        const int wzp = z == N2 - 1 ? w - (N2 - 1) * SZ : w + SZ;
        const int wzm = z == 0 ? w + (N2 - 1) * SZ : w - SZ;
        uint32_t nzp = nb[wzp], nzm = nb[wzm], jzm = Jz[wzm];
        if (z == N2 - 1)
            nzp = rot_zp(nzp);
        if (z == 0) {
            nzm = rot_zm(nzm);
            jzm = rot_zm(jzm);
        }
        return count6(s ^ nb[wxp] ^ Jx[w], s ^ nb[wxm] ^ Jx[wxm], s ^ nb[wyp] ^ Jy[w],
                      s ^ nb[wym] ^ Jy[wym], s ^ nzp ^ Jz[w], s ^ nzm ^ jzm);
    };
    tile_finish_at(jb, tb, w, s, M, M2, c2, upd, live0, live1, live2, always3, T1x, T0, c1, c3, rk,
                   calls, recount);
}

// Full adders of three bits: sum and carry.
__device__ __forceinline__ void add3(uint32_t a, uint32_t b, uint32_t c, uint32_t &sum,
                                     uint32_t &carry)
{
    sum = a ^ b ^ c;
    carry = maj3(a, b, c);
}

// One word of a tile: its outright flips (u >= 3) and whether the leading
// bits M of its first draws might accept a lane.  With LOWT the classes 1 and
// 0 are tested against the job's 32-lane bounds T1x, T0, a superset of the
// exact per-count test.
template <bool LOWT>
__device__ __forceinline__ bool tile_word(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3,
                                          uint32_t u4, uint32_t u5, uint32_t M,
                                          const TileTables &tb, uint32_t T1x, uint32_t T0,
                                          uint32_t live0, uint32_t live1, uint32_t live2,
                                          uint32_t &alw, uint32_t &m2)
{
    if (LOWT) {
        // u = 2 (k1 + k2) + s1 + s2 from two full adders
        uint32_t s1, k1, s2, k2;
        add3(u0, u1, u2, s1, k1);
        add3(u3, u4, u5, s2, k2);
        alw = maj3(k1, k2, s1 | s2);           // u >= 3
        m2 = (k1 | k2 | (s1 & s2)) & ~alw;     // u == 2
        return (M <= tb.lead[2][__popc(m2)]) | ((M & 0xFFC00u) <= T1x) | ((M & 0x3FFu) <= T0);
    } else {
        const Count c = count6(u0, u1, u2, u3, u4, u5);
        alw = c.b2 | (c.b1 & c.b0);
        const Classes k = classes(c, alw, 0xffffffffu, live0, live1, live2);
        m2 = k.M2;
        return (M <= tb.lead[2][__popc(k.M2)]) | ((M & 0xFFC00u) <= tb.lead[1][__popc(k.M1)]) |
               ((M & 0x3FFu) <= tb.lead[0][__popc(k.M0)]);
    }
}

template <bool COUNT, int MAXJ, int GL, bool LOWT>
__global__ void __launch_bounds__(kSweepThreads, 9)
    metro_tile_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    constexpr int N2 = GL / 32, SZ = GL * GL;
    constexpr int XP = GL / 2, ZP = N2 / 2;
    constexpr int XPLOG = GL == 128 ? 6 : 5;
    constexpr uint32_t W = (uint32_t)SZ * N2;
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    __shared__ TileTables tb;
    __shared__ uint4 s_q[kSweepThreads / 32][kTileQueue];
    __shared__ int s_qn[kSweepThreads / 32];
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33, n = i - 33 * u;
        const uint32_t hi = jb->gC_hi[u][n];
        tb.hi[u][n] = hi;
        tb.lead[u][n] = u == 2 ? lead2(hi) : u == 1 ? lead1(hi) : lead0(hi);
    }
    if (threadIdx.x < kSweepThreads / 32)
        s_qn[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;

    const int h = P.h;
    const int lane = threadIdx.x & 31;
    uint4 *q = s_q[threadIdx.x >> 5];
    int *qn = &s_qn[threadIdx.x >> 5];
    const int Y = G.seg;
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    const int tl = (local - s * G.bps) * kSweepThreads + (int)threadIdx.x;
    const int x0 = 2 * (tl & (XP - 1));
    const int z0 = 2 * ((tl >> XPLOG) & (ZP - 1));  // uniform over a warp (XP >= 32)
    // threads past the last segment of a row range (ea_set_row_range) run no
    // row; a warp is wholly in or out (a row of tiles is a whole number of warps)
    const bool act = (tl >> XPLOG) / ZP * Y < G.row_n;
    const int y0 = G.row0 + (act ? (tl >> XPLOG) / ZP * Y : 0);
    const int Yrun = act ? Y : 0;
    const bool all_always = (J.meta >> 3) & 1u, none_random = (J.meta >> 4) & 1u;
    const uint32_t live0 = 0u - (J.meta & 1u), live1 = 0u - ((J.meta >> 1) & 1u),
                   live2 = 0u - ((J.meta >> 2) & 1u);
    const uint32_t always3 = jb->always_u & 7u;
    const uint32_t T1x = lead1(jb->gC_hi[1][32]), T0 = lead0(jb->gC_hi[0][32]);
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2m = dev::kStreamMetropolis | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    const int oz0 = z0 * SZ, oz1 = oz0 + SZ;
    const int ozm = (z0 == 0 ? N2 - 1 : z0 - 1) * SZ;
    const int ozp = (z0 + 2 == N2 ? 0 : z0 + 2) * SZ;
    const bool wrap_m = z0 == 0, wrap_p = z0 + 2 == N2;
    const int xm = (x0 - 1) & (GL - 1), xq = (x0 + 2) & (GL - 1);
    unsigned int n_words = 0, n_calls = 0, n_extra = 0;

    // the window: neighbour rows y - 1 (m) and y (c), y bonds of row y - 1
    const int rym = ((y0 - 1) & (GL - 1)) * GL;
    uint2 Nm0 = ld2(nb, x0 + rym + oz0), Nm1 = ld2(nb, x0 + rym + oz1);
    uint2 Jym0 = ld2(Jy, x0 + rym + oz0), Jym1 = ld2(Jy, x0 + rym + oz1);
    uint2 Nc0 = ld2(nb, x0 + y0 * GL + oz0), Nc1 = ld2(nb, x0 + y0 * GL + oz1);
    for (int i = 0; i < Yrun; ++i) {
        const int y = y0 + i;
        const int ry = y * GL, ryp = ((y + 1) & (GL - 1)) * GL;
        const int w0 = x0 + ry + oz0, w1 = x0 + ry + oz1;  // the even-x words at z0, z0 + 1
        const uint2 S0 = ld2(upd, w0), S1 = ld2(upd, w1);
        const uint2 Nn0 = ld2(nb, x0 + ryp + oz0), Nn1 = ld2(nb, x0 + ryp + oz1);
        uint2 Nzm = ld2(nb, x0 + ry + ozm), Nzp = ld2(nb, x0 + ry + ozp);
        uint2 Jzm = ld2(Jz, x0 + ry + ozm);
        const uint32_t Xm0 = nb[xm + ry + oz0], Xm1 = nb[xm + ry + oz1];
        const uint32_t Xp0 = nb[xq + ry + oz0], Xp1 = nb[xq + ry + oz1];
        const uint32_t Jxm0 = Jx[xm + ry + oz0], Jxm1 = Jx[xm + ry + oz1];
        const uint2 Jx0 = ld2(Jx, w0), Jx1 = ld2(Jx, w1);
        const uint2 Jy0 = ld2(Jy, w0), Jy1 = ld2(Jy, w1);
        const uint2 Jz0 = ld2(Jz, w0), Jz1 = ld2(Jz, w1);
        if (wrap_m) {
            Nzm = make_uint2(rot_zm(Nzm.x), rot_zm(Nzm.y));
            Jzm = make_uint2(rot_zm(Jzm.x), rot_zm(Jzm.y));
        }
        if (wrap_p)
            Nzp = make_uint2(rot_zp(Nzp.x), rot_zp(Nzp.y));
        // main calls: pair (x0, z0 | z0 + 1) and pair (x0 + 1, z0 | z0 + 1)
        const uint32_t c2A = c2m | ((uint32_t)(h ^ (y & 1)) << 11);
        uint4 R = make_uint4(0u, 0u, 0u, 0u);
        if (!(all_always || none_random))  // the quad's main call
            R = dev::philox10_rk(make_uint4((uint32_t)w0, c1, c2A, c3), rk);
        // words a0 = (x0, z0), a1 = (x0 + 1, z0), b0 = (x0, z0 + 1), b1 = (x0 + 1, z0 + 1)
        uint32_t alwa0, alwa1, alwb0, alwb1, m2a0, m2a1, m2b0, m2b1;
        uint32_t sp = S0.x;
        const bool draw = !(all_always || none_random);
        bool ha0 = tile_word<LOWT>(sp ^ Nc0.y ^ Jx0.x, sp ^ Xm0 ^ Jxm0, sp ^ Nn0.x ^ Jy0.x,
                                   sp ^ Nm0.x ^ Jym0.x, sp ^ Nc1.x ^ Jz0.x, sp ^ Nzm.x ^ Jzm.x,
                                   R.x, tb, T1x, T0, live0, live1, live2, alwa0, m2a0);
        sp = S0.y;
        bool ha1 = tile_word<LOWT>(sp ^ Xp0 ^ Jx0.y, sp ^ Nc0.x ^ Jx0.x, sp ^ Nn0.y ^ Jy0.y,
                                   sp ^ Nm0.y ^ Jym0.y, sp ^ Nc1.y ^ Jz0.y, sp ^ Nzm.y ^ Jzm.y,
                                   R.y, tb, T1x, T0, live0, live1, live2, alwa1, m2a1);
        sp = S1.x;
        bool hb0 = tile_word<LOWT>(sp ^ Nc1.y ^ Jx1.x, sp ^ Xm1 ^ Jxm1, sp ^ Nn1.x ^ Jy1.x,
                                   sp ^ Nm1.x ^ Jym1.x, sp ^ Nzp.x ^ Jz1.x, sp ^ Nc0.x ^ Jz0.x,
                                   R.z, tb, T1x, T0, live0, live1, live2, alwb0, m2b0);
        sp = S1.y;
        bool hb1 = tile_word<LOWT>(sp ^ Xp1 ^ Jx1.y, sp ^ Nc1.x ^ Jx1.x, sp ^ Nn1.y ^ Jy1.y,
                                   sp ^ Nm1.y ^ Jym1.y, sp ^ Nzp.y ^ Jz1.y, sp ^ Nc0.y ^ Jz0.y,
                                   R.w, tb, T1x, T0, live0, live1, live2, alwb1, m2b1);
        ha0 = ha0 && draw;
        ha1 = ha1 && draw;
        hb0 = hb0 && draw;
        hb1 = hb1 && draw;
        Nm0 = Nc0;
        Nm1 = Nc1;
        Nc0 = Nn0;
        Nc1 = Nn1;
        Jym0 = Jy0;
        Jym1 = Jy1;
        // every word is written with its outright flips; a queued word is
        // written again by the rare path
        const uint32_t fx = all_always ? 0xffffffffu : 0u;
        *reinterpret_cast<uint2 *>(upd + w0) = make_uint2(S0.x ^ (alwa0 | fx), S0.y ^ (alwa1 | fx));
        *reinterpret_cast<uint2 *>(upd + w1) = make_uint2(S1.x ^ (alwb0 | fx), S1.y ^ (alwb1 | fx));
        if (COUNT)
            n_words += 4;
        if (all_always || none_random)
            continue;
        if (COUNT)
            n_calls += 1;
        if (ha0)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w0, S0.x, R.x, m2a0);
        if (ha1)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w0 + 1u, S0.y, R.y, m2a1);
        if (hb0)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w1, S1.x, R.z, m2b0);
        if (hb1)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w1 + 1u, S1.y, R.w, m2b1);
        __syncwarp();
        int q_n = *qn;
        if (q_n >= 96) {  // full rounds, one queued word per lane, while 32 are queued
            do {
                q_n -= 32;
                const uint4 e = q[q_n + lane];
                unsigned int extra = 0;
                tile_finish<GL>(jb, tb, e, upd, nb, Jx, Jy, Jz, h, live0, live1, live2, always3,
                                T1x, T0, c1, c2m, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
            } while (q_n >= 32);
            if (lane == 0)
                *qn = q_n;
            __syncwarp();
        }
    }
    // the words still queued in the block's four warps, pooled and shared out
    // in rounds of 32 over the warps
    __syncthreads();
    const int n0q = s_qn[0], n1q = n0q + s_qn[1], n2q = n1q + s_qn[2], n3q = n2q + s_qn[3];
    for (int g = (int)threadIdx.x; g < n3q; g += kSweepThreads) {
        const int wq = g < n0q ? 0 : g < n1q ? 1 : g < n2q ? 2 : 3;
        const int off = g - (wq == 0 ? 0 : wq == 1 ? n0q : wq == 2 ? n1q : n2q);
        unsigned int extra = 0;
        tile_finish<GL>(jb, tb, s_q[wq][off], upd, nb, Jx, Jy, Jz, h, live0, live1, live2, always3,
                        T1x, T0, c1, c2m, c3, rk, extra);
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_calls + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// ---------------------------------------------------------------------------
// Metropolis half-step for side 128 with the rows staged in shared memory.
// A block of 128 threads owns the whole xz plane of the word lattice (128 x 4
// words, thread (x pair, z pair) as in metro_tile_kernel) over a segment of Y
// rows along y.  One warp's lanes bring each row's words into shared memory
// with bulk asynchronous copies (cp.async.bulk, the TMA engine): row y + 1 of
// the updated area and of the three coupling arrays and row y + 2 of the
// neighbour area are in flight while row y is computed, and complete on an
// mbarrier.  The threads then read every word with shared-memory loads:
// no global-memory latency on the stencil.  Ring buffers: 4 neighbour rows
// (y - 1, y, y + 1 in use, y + 2 in flight), 3 rows of y bonds, 2 of the
// updated area and of the x and z bonds.
// The rare path is split: words whose class dE = 4 alone might flip (nearly
// all) are finished by a short routine on the full 64-bit draws; words whose
// classes dE = 8 or 12 might flip go to tile_finish_at.  The draws are those
// of every other Metropolis kernel.
// Every wait on a barrier is bounded (P.wait_limit polls); when one runs out
// the block waits for its own copies still in flight, records the timeout in
// the device status word and returns.
// ---------------------------------------------------------------------------
constexpr int kStageRow = 512;     // words of one row of the xz plane at side 128
constexpr int kStageQueue = 160;   // entries per warp: up to 31 left + 128 per row
constexpr int kStageHeavy = 64;    // entries per warp whose dE = 8 or 12 leads hit
constexpr uint32_t kStageGroupBytes = 5 * kStageRow * 4;  // one row of five arrays
constexpr uint32_t kStageFirstBytes = 8 * kStageRow * 4;  // the first group: 8 rows
constexpr uint32_t kDrainPolls = 1u << 24;

__device__ unsigned int g_sweep_status;  // bit 0: a bounded wait ran out

struct StageSmem {
    uint32_t nb[4][kStageRow];
    uint32_t jy[3][kStageRow];
    uint32_t up[2][kStageRow];
    uint32_t jx[2][kStageRow];
    uint32_t jz[2][kStageRow];
    uint64_t bar[2];
    uint64_t bar_never;  // nothing ever arrives on it (the timeout test waits on it)
    uint4 q[kSweepThreads / 32][kStageQueue];
    uint4 hq[kSweepThreads / 32][kStageHeavy];
    int qn[kSweepThreads / 32], hn[kSweepThreads / 32];
    uint32_t c2hi[33], c2lo[33];  // C_2[g] (class dE = 4), full 64 bits
    TileTables tb;
};

__device__ __forceinline__ uint2 lds2(const uint32_t *p)
{
    return *reinterpret_cast<const uint2 *>(p);
}

// The short rare path of a queued word e = (word-site, spins, main bits M,
// class-2 lanes) whose classes dE = 8 and 12 select nothing: class dE = 4 by
// geometric gaps on full 64-bit draws (draw 0 completed by extension call 64,
// draws d >= 1 from calls 3 + 3 ((d - 1) div 2)).  The word was stored with its
// outright flips; that value is read back and the accepted lanes added.
__device__ __forceinline__ void stage_finish(const StageSmem &S, const uint4 &e,
                                             uint32_t *__restrict__ upd, int h, uint32_t c1,
                                             uint32_t c2m, uint32_t c3,
                                             const uint32_t (&rk)[20], unsigned int &calls)
{
    const int w = (int)e.x;
    const uint32_t M = e.z;
    const int x = w & 127, y = (w >> 7) & 127, z = w >> 14;
    const uint32_t c2 = c2m | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
    const uint32_t base = upd[w];
    const uint4 X = dev::philox10_rk(make_uint4((uint32_t)w, c1, c2 | 64u, c3), rk);
    ++calls;
    auto C = [&S](int g) -> uint64_t { return ((uint64_t)S.c2hi[g] << 32) | S.c2lo[g]; };
    uint64_t V = first_draw2(M, X);
    uint32_t Mr = e.w, A = 0u;
    int rem = __popc(Mr), d = 0;
    uint4 Q = make_uint4(0u, 0u, 0u, 0u);
    while (rem > 0 && V < C(rem)) {
        // G = min{g : V < C[g + 1]} by bisection over the nondecreasing table
        int lo = 1, hi = rem;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (V < C(mid))
                hi = mid;
            else
                lo = mid + 1;
        }
        const int G = lo - 1;
        const uint32_t bit = nth_bit(Mr, G);
        A |= bit;
        Mr &= ~(bit | (bit - 1u));
        rem -= G + 1;
        if (rem == 0)
            break;
        ++d;
        if (((d - 1) & 1) == 0) {
            Q = dev::philox10_rk(
                make_uint4((uint32_t)w, c1, c2 | (uint32_t)(3 + 3 * ((d - 1) >> 1)), c3), rk);
            ++calls;
        }
        V = ((d - 1) & 1) ? (((uint64_t)Q.z << 32) | Q.w) : (((uint64_t)Q.x << 32) | Q.y);
    }
    if (A)
        upd[w] = base ^ A;
}

template <bool COUNT, int MAXJ>
__global__ void __launch_bounds__(kSweepThreads, 5)
    metro_stage_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    constexpr int GL = 128, N2 = 4, SZ = GL * GL;
    constexpr uint32_t W = (uint32_t)SZ * N2;
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    __shared__ StageSmem S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;  // this job has stopped (uniform over the block)
    const int h = P.h;
    const int Y = G.seg;
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    const int y0 = G.row0 + (local - s * G.bps) * Y;
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;

    // the first group: rows y0 of the updated area and of the x, z bonds, y bonds
    // of rows y0 - 1 and y0, neighbour rows y0 - 1 .. y0 + 1; one copy per lane
    // of warp 0 (a row of one array is four 512-byte runs, one per z')
    if (threadIdx.x == 0) {
        dev::mbar_init(&S.bar[0], 1);
        dev::mbar_init(&S.bar[1], 1);
        dev::mbar_init(&S.bar_never, 1);
        dev::mbar_init_fence();
    }
    __syncthreads();
    auto row_src = [&](const uint32_t *a, int y, int zq) {
        return a + (size_t)((y & (GL - 1)) * GL + zq * SZ);
    };
    if (warp == 0) {
        if (lane == 0)
            dev::mbar_arrive_expect_tx(&S.bar[0], kStageFirstBytes);
        __syncwarp();
        const int a = lane >> 2, zq = lane & 3;
        const uint32_t *src;
        uint32_t *dst;
        switch (a) {
        case 0: src = row_src(upd, y0, zq); dst = S.up[0]; break;
        case 1: src = row_src(Jx, y0, zq); dst = S.jx[0]; break;
        case 2: src = row_src(Jz, y0, zq); dst = S.jz[0]; break;
        case 3: src = row_src(Jy, y0 - 1, zq); dst = S.jy[0]; break;
        case 4: src = row_src(Jy, y0, zq); dst = S.jy[1]; break;
        case 5: src = row_src(nb, y0 - 1, zq); dst = S.nb[0]; break;
        case 6: src = row_src(nb, y0, zq); dst = S.nb[1]; break;
        default: src = row_src(nb, y0 + 1, zq); dst = S.nb[2]; break;
        }
        dev::bulk_g2s(dst + zq * GL, src, GL * 4, &S.bar[0]);
    }

    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33, n = i - 33 * u;
        const uint32_t hi = jb->gC_hi[u][n];
        S.tb.hi[u][n] = hi;
        S.tb.lead[u][n] = u == 2 ? lead2(hi) : u == 1 ? lead1(hi) : lead0(hi);
        if (u == 2) {
            S.c2hi[n] = hi;
            S.c2lo[n] = jb->gC_lo[2][n];
        }
    }
    if (lane == 0) {
        S.qn[warp] = 0;
        S.hn[warp] = 0;
    }
    const int xp = threadIdx.x & 63, zp = threadIdx.x >> 6;
    const int x0 = 2 * xp, z0 = 2 * zp;
    const int po = z0 * GL + x0, po1 = po + GL;  // the thread's pair at z0, z0 + 1 in a row
    const bool wrap_m = z0 == 0, wrap_p = z0 + 2 == N2;
    const int zmo = (wrap_m ? N2 - 1 : z0 - 1) * GL + x0, zpo = (wrap_p ? 0 : z0 + 2) * GL + x0;
    const int xm = (x0 - 1) & (GL - 1), xq = (x0 + 2) & (GL - 1);
    const int xmo0 = z0 * GL + xm, xmo1 = xmo0 + GL, xqo0 = z0 * GL + xq, xqo1 = xqo0 + GL;
    const bool none_random = (J.meta >> 4) & 1u;
    const uint32_t live0 = 0u - (J.meta & 1u), live1 = 0u - ((J.meta >> 1) & 1u),
                   live2 = 0u - ((J.meta >> 2) & 1u);
    const uint32_t always3 = jb->always_u & 7u;
    const uint32_t T1x = lead1(jb->gC_hi[1][32]), T0 = lead0(jb->gC_hi[0][32]);
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2m = dev::kStreamMetropolis | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    uint4 *q = S.q[warp];
    uint4 *hq = S.hq[warp];
    unsigned int n_words = 0, n_calls = 0, n_extra = 0;
    // P.wait_mode bit 0 (tests of the timeout path only): wait on a barrier that no
    // copy completes, so that the bounded wait runs out
    uint64_t *const wait_bar_test = (P.wait_mode & 1u) ? &S.bar_never : nullptr;

    for (int i = 0; i < Y; ++i) {
        const int y = y0 + i;
        // (a) this row's group has landed; (b) every thread is past row i - 1
        const bool ok = wait_bar_test ? dev::mbar_wait_bounded(wait_bar_test, 0u, P.wait_limit)
                                      : dev::mbar_wait_bounded(&S.bar[i & 1], (i >> 1) & 1,
                                                               P.wait_limit);
        if (__syncthreads_or(!ok)) {
            dev::mbar_wait_bounded(&S.bar[i & 1], (i >> 1) & 1, kDrainPolls);
            if (threadIdx.x == 0)
                atomicOr(&g_sweep_status, 1u);
            return;
        }
        // (c) the next row's group, into the slots row i - 1 has released
        if (i + 1 < Y && warp == 0) {
            const int k = (i + 1) & 1;
            if (lane == 0)
                dev::mbar_arrive_expect_tx(&S.bar[k], kStageGroupBytes);
            __syncwarp();
            if (lane < 20) {
                dev::fence_proxy_async_smem();
                const int a = lane >> 2, zq = lane & 3;
                const uint32_t *src;
                uint32_t *dst;
                switch (a) {
                case 0: src = row_src(upd, y + 1, zq); dst = S.up[k]; break;
                case 1: src = row_src(Jx, y + 1, zq); dst = S.jx[k]; break;
                case 2: src = row_src(Jz, y + 1, zq); dst = S.jz[k]; break;
                case 3: src = row_src(Jy, y + 1, zq); dst = S.jy[(i + 2) % 3]; break;
                default: src = row_src(nb, y + 2, zq); dst = S.nb[(i + 3) & 3]; break;
                }
                dev::bulk_g2s(dst + zq * GL, src, GL * 4, &S.bar[k]);
            }
        }
        // (d) row y from shared memory
        const uint32_t *nbc = S.nb[(i + 1) & 3], *nbm = S.nb[i & 3], *nbn = S.nb[(i + 2) & 3];
        const uint32_t *jyc = S.jy[(i + 1) % 3], *jym = S.jy[i % 3];
        const uint32_t *sup = S.up[i & 1], *sjx = S.jx[i & 1], *sjz = S.jz[i & 1];
        const uint2 S0 = lds2(sup + po), S1 = lds2(sup + po1);
        const uint2 Nc0 = lds2(nbc + po), Nc1 = lds2(nbc + po1);
        const uint2 Nm0 = lds2(nbm + po), Nm1 = lds2(nbm + po1);
        const uint2 Nn0 = lds2(nbn + po), Nn1 = lds2(nbn + po1);
        uint2 Nzm = lds2(nbc + zmo), Nzp = lds2(nbc + zpo);
        const uint32_t Xm0 = nbc[xmo0], Xm1 = nbc[xmo1], Xp0 = nbc[xqo0], Xp1 = nbc[xqo1];
        const uint2 Jx0 = lds2(sjx + po), Jx1 = lds2(sjx + po1);
        const uint32_t Jxm0 = sjx[xmo0], Jxm1 = sjx[xmo1];
        const uint2 Jy0 = lds2(jyc + po), Jy1 = lds2(jyc + po1);
        const uint2 Jym0 = lds2(jym + po), Jym1 = lds2(jym + po1);
        const uint2 Jz0 = lds2(sjz + po), Jz1 = lds2(sjz + po1);
        uint2 Jzm = lds2(sjz + zmo);
        if (wrap_m) {
            Nzm = make_uint2(rot_zm(Nzm.x), rot_zm(Nzm.y));
            Jzm = make_uint2(rot_zm(Jzm.x), rot_zm(Jzm.y));
        }
        if (wrap_p)
            Nzp = make_uint2(rot_zp(Nzp.x), rot_zp(Nzp.y));
        const int w0 = x0 + y * GL + z0 * SZ, w1 = w0 + SZ;
        const uint32_t c2A = c2m | ((uint32_t)(h ^ (y & 1)) << 11);
        uint4 R = make_uint4(0u, 0u, 0u, 0u);
        if (!none_random)
            R = dev::philox10_rk(make_uint4((uint32_t)w0, c1, c2A, c3), rk);
        uint32_t alwa0, alwa1, alwb0, alwb1, m2a0, m2a1, m2b0, m2b1;
        uint32_t sp = S0.x;
        bool ha0 = tile_word<true>(sp ^ Nc0.y ^ Jx0.x, sp ^ Xm0 ^ Jxm0, sp ^ Nn0.x ^ Jy0.x,
                                   sp ^ Nm0.x ^ Jym0.x, sp ^ Nc1.x ^ Jz0.x, sp ^ Nzm.x ^ Jzm.x,
                                   R.x, S.tb, T1x, T0, live0, live1, live2, alwa0, m2a0);
        sp = S0.y;
        bool ha1 = tile_word<true>(sp ^ Xp0 ^ Jx0.y, sp ^ Nc0.x ^ Jx0.x, sp ^ Nn0.y ^ Jy0.y,
                                   sp ^ Nm0.y ^ Jym0.y, sp ^ Nc1.y ^ Jz0.y, sp ^ Nzm.y ^ Jzm.y,
                                   R.y, S.tb, T1x, T0, live0, live1, live2, alwa1, m2a1);
        sp = S1.x;
        bool hb0 = tile_word<true>(sp ^ Nc1.y ^ Jx1.x, sp ^ Xm1 ^ Jxm1, sp ^ Nn1.x ^ Jy1.x,
                                   sp ^ Nm1.x ^ Jym1.x, sp ^ Nzp.x ^ Jz1.x, sp ^ Nc0.x ^ Jz0.x,
                                   R.z, S.tb, T1x, T0, live0, live1, live2, alwb0, m2b0);
        sp = S1.y;
        bool hb1 = tile_word<true>(sp ^ Xp1 ^ Jx1.y, sp ^ Nc1.x ^ Jx1.x, sp ^ Nn1.y ^ Jy1.y,
                                   sp ^ Nm1.y ^ Jym1.y, sp ^ Nzp.y ^ Jz1.y, sp ^ Nc0.y ^ Jz0.y,
                                   R.w, S.tb, T1x, T0, live0, live1, live2, alwb1, m2b1);
        *reinterpret_cast<uint2 *>(upd + w0) = make_uint2(S0.x ^ alwa0, S0.y ^ alwa1);
        *reinterpret_cast<uint2 *>(upd + w1) = make_uint2(S1.x ^ alwb0, S1.y ^ alwb1);
        if (COUNT)
            n_words += 4;
        if (none_random)
            continue;
        if (COUNT)
            n_calls += 1;
        if (ha0)
            q[atomicAdd(&S.qn[warp], 1)] = make_uint4((uint32_t)w0, S0.x, R.x, m2a0);
        if (ha1)
            q[atomicAdd(&S.qn[warp], 1)] = make_uint4((uint32_t)w0 + 1u, S0.y, R.y, m2a1);
        if (hb0)
            q[atomicAdd(&S.qn[warp], 1)] = make_uint4((uint32_t)w1, S1.x, R.z, m2b0);
        if (hb1)
            q[atomicAdd(&S.qn[warp], 1)] = make_uint4((uint32_t)w1 + 1u, S1.y, R.w, m2b1);
        __syncwarp();
        int q_n = S.qn[warp];
        while (q_n >= 32) {  // rounds of one queued word per lane
            q_n -= 32;
            const uint4 e = q[q_n + lane];
            const bool heavy = ((e.z & 0xFFC00u) <= T1x) | ((e.z & 0x3FFu) <= T0) | (always3 != 0u);
            const uint32_t hv = __ballot_sync(0xffffffffu, heavy);
            const int hn = S.hn[warp];
            if (heavy)
                hq[hn + __popc(hv & ((1u << lane) - 1u))] = e;
            else {
                unsigned int extra = 0;
                stage_finish(S, e, upd, h, c1, c2m, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
            }
            __syncwarp();
            if (lane == 0)
                S.hn[warp] = hn + __popc(hv);
            __syncwarp();
            if (S.hn[warp] >= 32) {  // a round of the words with dE = 8 or 12 leads
                const int k = S.hn[warp] - 32;
                unsigned int extra = 0;
                tile_finish<GL>(jb, S.tb, hq[k + lane], upd, nb, Jx, Jy, Jz, h, live0, live1,
                                live2, always3, T1x, T0, c1, c2m, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
                if (lane == 0)
                    S.hn[warp] = k;
                __syncwarp();
            }
        }
        if (lane == 0)
            S.qn[warp] = q_n;
        __syncwarp();
    }
    // the words still queued in the block's four warps, pooled and shared out
    __syncthreads();
    int nq[5] = {0, 0, 0, 0, 0}, nh[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nq[k + 1] = nq[k] + S.qn[k];
        nh[k + 1] = nh[k] + S.hn[k];
    }
    for (int g = (int)threadIdx.x; g < nq[4] + nh[4]; g += kSweepThreads) {
        unsigned int extra = 0;
        if (g < nq[4]) {
            const int wq = g < nq[1] ? 0 : g < nq[2] ? 1 : g < nq[3] ? 2 : 3;
            const uint4 e = S.q[wq][g - nq[wq]];
            const bool heavy = ((e.z & 0xFFC00u) <= T1x) | ((e.z & 0x3FFu) <= T0) | (always3 != 0u);
            if (heavy)
                tile_finish<GL>(jb, S.tb, e, upd, nb, Jx, Jy, Jz, h, live0, live1, live2, always3,
                                T1x, T0, c1, c2m, c3, rk, extra);
            else
                stage_finish(S, e, upd, h, c1, c2m, c3, rk, extra);
        } else {
            const int gh = g - nq[4];
            const int wq = gh < nh[1] ? 0 : gh < nh[2] ? 1 : gh < nh[3] ? 2 : 3;
            tile_finish<GL>(jb, S.tb, S.hq[wq][gh - nh[wq]], upd, nb, Jx, Jy, Jz, h, live0, live1,
                            live2, always3, T1x, T0, c1, c2m, c3, rk, extra);
        }
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_calls + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// ---------------------------------------------------------------------------
// Metropolis half-step for jobs whose 32 lanes all lie along y and z (kx = 1:
// the sides divisible by 16) other than 64 and 128.  The tiles, window and
// queue of metro_tile_kernel, with the word lattice n0 x n1 x n2 read at run
// time: a thread owns (x0, x0 + 1) x (z0, z0 + 1) over a segment of Y rows
// (Y divides n1, so a segment never crosses the y wrap); the neighbour word
// read across the y or z wrap is realigned lane by lane, the x wrap needs no
// realignment.  Threads past the sample's last tile run on a valid tile and
// write nothing.
// ---------------------------------------------------------------------------
struct GTileGeo {
    int n0, n1, n2;
    Axis ay, az;
};

// The class count of word w (spins s, at (x, y, z)) from the neighbour area,
// with the y and z wraps realigned.
__device__ __forceinline__ Count gtile_count(int w, uint32_t s, int x, int y, int z,
                                             const uint32_t *__restrict__ nb,
                                             const uint32_t *__restrict__ Jx,
                                             const uint32_t *__restrict__ Jy,
                                             const uint32_t *__restrict__ Jz, const GTileGeo &gg)
{
    const int n0 = gg.n0, n1 = gg.n1, n2 = gg.n2, sz = n0 * n1;
    const int wxp = x == n0 - 1 ? w - (n0 - 1) : w + 1;
    const int wxm = x == 0 ? w + (n0 - 1) : w - 1;
    const int wyp = y == n1 - 1 ? w - (n1 - 1) * n0 : w + n0;
    const int wym = y == 0 ? w + (n1 - 1) * n0 : w - n0;
    const int wzp = z == n2 - 1 ? w - (n2 - 1) * sz : w + sz;
    const int wzm = z == 0 ? w + (n2 - 1) * sz : w - sz;
    uint32_t nyp = nb[wyp], nym = nb[wym], jym = Jy[wym];
    uint32_t nzp = nb[wzp], nzm = nb[wzm], jzm = Jz[wzm];
    if (y == n1 - 1)
        nyp = fixup(nyp, gg.ay, 0);
    if (y == 0) {
        nym = fixup(nym, gg.ay, 1);
        jym = fixup(jym, gg.ay, 1);
    }
    if (z == n2 - 1)
        nzp = fixup(nzp, gg.az, 0);
    if (z == 0) {
        nzm = fixup(nzm, gg.az, 1);
        jzm = fixup(jzm, gg.az, 1);
    }
    return count6(s ^ nb[wxp] ^ Jx[w], s ^ nb[wxm] ^ Jx[wxm], s ^ nyp ^ Jy[w], s ^ nym ^ jym,
                  s ^ nzp ^ Jz[w], s ^ nzm ^ jzm);
}

__device__ __forceinline__ void gtile_finish(const JobDev *__restrict__ jb, const TileTables &tb,
                                             const uint4 &e, uint32_t *__restrict__ upd,
                                             const uint32_t *__restrict__ nb,
                                             const uint32_t *__restrict__ Jx,
                                             const uint32_t *__restrict__ Jy,
                                             const uint32_t *__restrict__ Jz, const GTileGeo &gg,
                                             int h, uint32_t live0, uint32_t live1, uint32_t live2,
                                             uint32_t always3, uint32_t T1x, uint32_t T0,
                                             uint32_t c1, uint32_t c2m, uint32_t c3,
                                             const uint32_t (&rk)[20], unsigned int &calls)
{
    const int n0 = gg.n0, n1 = gg.n1;
    const int w = (int)e.x;
    const uint32_t s = e.y, M = e.z, M2 = e.w;
    const int x = w % n0, r = w / n0, y = r % n1, z = r / n1;
    const uint32_t c2 = c2m | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
    const auto recount = [&]() -> Count { return gtile_count(w, s, x, y, z, nb, Jx, Jy, Jz, gg); };
    tile_finish_at(jb, tb, w, s, M, M2, c2, upd, live0, live1, live2, always3, T1x, T0, c1, c3, rk,
                   calls, recount);
}

template <bool COUNT, int MAXJ, bool LOWT>
__global__ void __launch_bounds__(kSweepThreads, 8)
    metro_gtile_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    __shared__ TileTables tb;
    __shared__ uint4 s_q[kSweepThreads / 32][kTileQueue];
    __shared__ int s_qn[kSweepThreads / 32];
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33, n = i - 33 * u;
        const uint32_t hi = jb->gC_hi[u][n];
        tb.hi[u][n] = hi;
        tb.lead[u][n] = u == 2 ? lead2(hi) : u == 1 ? lead1(hi) : lead0(hi);
    }
    if (threadIdx.x < kSweepThreads / 32)
        s_qn[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;

    const int h = P.h;
    const int lane = threadIdx.x & 31;
    uint4 *q = s_q[threadIdx.x >> 5];
    int *qn = &s_qn[threadIdx.x >> 5];
    GTileGeo gg;
    gg.n0 = G.n0;
    gg.n1 = G.n1;
    gg.n2 = G.n2;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        gg.ay.sA[dir] = G.ysA[dir];
        gg.ay.sB[dir] = G.ysB[dir];
        gg.ay.mA[dir] = G.ymA[dir];
        gg.ay.mB[dir] = G.ymB[dir];
        gg.az.sA[dir] = G.zsA[dir];
        gg.az.sB[dir] = G.zsB[dir];
        gg.az.mA[dir] = G.zmA[dir];
        gg.az.mB[dir] = G.zmB[dir];
    }
    const int n0 = gg.n0, n1 = gg.n1, n2 = gg.n2, SZ = n0 * n1;
    const int XP = n0 >> 1, ZP = n2 >> 1, Y = G.seg;
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    int tl = (local - s * G.bps) * kSweepThreads + (int)threadIdx.x;
    const bool act = tl < XP * ZP * (n1 / Y);
    if (!act)
        tl = 0;
    const int x0 = 2 * (tl % XP);
    const int z0 = 2 * ((tl / XP) % ZP);
    const int y0 = tl / XP / ZP * Y;
    const bool all_always = (J.meta >> 3) & 1u, none_random = (J.meta >> 4) & 1u;
    const uint32_t live0 = 0u - (J.meta & 1u), live1 = 0u - ((J.meta >> 1) & 1u),
                   live2 = 0u - ((J.meta >> 2) & 1u);
    const uint32_t always3 = jb->always_u & 7u;
    const uint32_t T1x = lead1(jb->gC_hi[1][32]), T0 = lead0(jb->gC_hi[0][32]);
    const uint32_t W = G.words;
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2m = dev::kStreamMetropolis | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    const int oz0 = z0 * SZ, oz1 = oz0 + SZ;
    const int ozm = (z0 == 0 ? n2 - 1 : z0 - 1) * SZ;
    const int ozp = (z0 + 2 == n2 ? 0 : z0 + 2) * SZ;
    const bool wrap_m = z0 == 0, wrap_p = z0 + 2 == n2;
    const int xm = x0 == 0 ? n0 - 1 : x0 - 1, xq = x0 + 2 == n0 ? 0 : x0 + 2;
    unsigned int n_words = 0, n_calls = 0, n_extra = 0;

    // the window: neighbour rows y - 1 (m) and y (c), y bonds of row y - 1; the
    // row above a segment that starts at y = 0 lies across the y wrap
    const int rym = (y0 == 0 ? n1 - 1 : y0 - 1) * n0;
    uint2 Nm0 = ld2(nb, x0 + rym + oz0), Nm1 = ld2(nb, x0 + rym + oz1);
    uint2 Jym0 = ld2(Jy, x0 + rym + oz0), Jym1 = ld2(Jy, x0 + rym + oz1);
    if (y0 == 0) {
        Nm0 = make_uint2(fixup(Nm0.x, gg.ay, 1), fixup(Nm0.y, gg.ay, 1));
        Nm1 = make_uint2(fixup(Nm1.x, gg.ay, 1), fixup(Nm1.y, gg.ay, 1));
        Jym0 = make_uint2(fixup(Jym0.x, gg.ay, 1), fixup(Jym0.y, gg.ay, 1));
        Jym1 = make_uint2(fixup(Jym1.x, gg.ay, 1), fixup(Jym1.y, gg.ay, 1));
    }
    uint2 Nc0 = ld2(nb, x0 + y0 * n0 + oz0), Nc1 = ld2(nb, x0 + y0 * n0 + oz1);
    for (int i = 0; i < Y; ++i) {
        const int y = y0 + i;
        const bool wrap_y = y + 1 == n1;  // only on a segment's last row
        const int ry = y * n0, ryp = wrap_y ? 0 : ry + n0;
        const int w0 = x0 + ry + oz0, w1 = x0 + ry + oz1;  // the even-x words at z0, z0 + 1
        const uint2 S0 = ld2(upd, w0), S1 = ld2(upd, w1);
        uint2 Nn0 = ld2(nb, x0 + ryp + oz0), Nn1 = ld2(nb, x0 + ryp + oz1);
        if (wrap_y) {
            Nn0 = make_uint2(fixup(Nn0.x, gg.ay, 0), fixup(Nn0.y, gg.ay, 0));
            Nn1 = make_uint2(fixup(Nn1.x, gg.ay, 0), fixup(Nn1.y, gg.ay, 0));
        }
        uint2 Nzm = ld2(nb, x0 + ry + ozm), Nzp = ld2(nb, x0 + ry + ozp);
        uint2 Jzm = ld2(Jz, x0 + ry + ozm);
        const uint32_t Xm0 = nb[xm + ry + oz0], Xm1 = nb[xm + ry + oz1];
        const uint32_t Xp0 = nb[xq + ry + oz0], Xp1 = nb[xq + ry + oz1];
        const uint32_t Jxm0 = Jx[xm + ry + oz0], Jxm1 = Jx[xm + ry + oz1];
        const uint2 Jx0 = ld2(Jx, w0), Jx1 = ld2(Jx, w1);
        const uint2 Jy0 = ld2(Jy, w0), Jy1 = ld2(Jy, w1);
        const uint2 Jz0 = ld2(Jz, w0), Jz1 = ld2(Jz, w1);
        if (wrap_m) {
            Nzm = make_uint2(fixup(Nzm.x, gg.az, 1), fixup(Nzm.y, gg.az, 1));
            Jzm = make_uint2(fixup(Jzm.x, gg.az, 1), fixup(Jzm.y, gg.az, 1));
        }
        if (wrap_p)
            Nzp = make_uint2(fixup(Nzp.x, gg.az, 0), fixup(Nzp.y, gg.az, 0));
        const uint32_t c2A = c2m | ((uint32_t)(h ^ (y & 1)) << 11);
        uint4 R = make_uint4(0u, 0u, 0u, 0u);
        if (!(all_always || none_random))  // the quad's main call
            R = dev::philox10_rk(make_uint4((uint32_t)w0, c1, c2A, c3), rk);
        uint32_t alwa0, alwa1, alwb0, alwb1, m2a0, m2a1, m2b0, m2b1;
        uint32_t sp = S0.x;
        const bool draw = act && !(all_always || none_random);
        bool ha0 = tile_word<LOWT>(sp ^ Nc0.y ^ Jx0.x, sp ^ Xm0 ^ Jxm0, sp ^ Nn0.x ^ Jy0.x,
                                   sp ^ Nm0.x ^ Jym0.x, sp ^ Nc1.x ^ Jz0.x, sp ^ Nzm.x ^ Jzm.x,
                                   R.x, tb, T1x, T0, live0, live1, live2, alwa0, m2a0);
        sp = S0.y;
        bool ha1 = tile_word<LOWT>(sp ^ Xp0 ^ Jx0.y, sp ^ Nc0.x ^ Jx0.x, sp ^ Nn0.y ^ Jy0.y,
                                   sp ^ Nm0.y ^ Jym0.y, sp ^ Nc1.y ^ Jz0.y, sp ^ Nzm.y ^ Jzm.y,
                                   R.y, tb, T1x, T0, live0, live1, live2, alwa1, m2a1);
        sp = S1.x;
        bool hb0 = tile_word<LOWT>(sp ^ Nc1.y ^ Jx1.x, sp ^ Xm1 ^ Jxm1, sp ^ Nn1.x ^ Jy1.x,
                                   sp ^ Nm1.x ^ Jym1.x, sp ^ Nzp.x ^ Jz1.x, sp ^ Nc0.x ^ Jz0.x,
                                   R.z, tb, T1x, T0, live0, live1, live2, alwb0, m2b0);
        sp = S1.y;
        bool hb1 = tile_word<LOWT>(sp ^ Xp1 ^ Jx1.y, sp ^ Nc1.x ^ Jx1.x, sp ^ Nn1.y ^ Jy1.y,
                                   sp ^ Nm1.y ^ Jym1.y, sp ^ Nzp.y ^ Jz1.y, sp ^ Nc0.y ^ Jz0.y,
                                   R.w, tb, T1x, T0, live0, live1, live2, alwb1, m2b1);
        ha0 = ha0 && draw;
        ha1 = ha1 && draw;
        hb0 = hb0 && draw;
        hb1 = hb1 && draw;
        Nm0 = Nc0;
        Nm1 = Nc1;
        Nc0 = Nn0;
        Nc1 = Nn1;
        Jym0 = Jy0;
        Jym1 = Jy1;
        const uint32_t fx = all_always ? 0xffffffffu : 0u;
        if (act) {
            *reinterpret_cast<uint2 *>(upd + w0) =
                make_uint2(S0.x ^ (alwa0 | fx), S0.y ^ (alwa1 | fx));
            *reinterpret_cast<uint2 *>(upd + w1) =
                make_uint2(S1.x ^ (alwb0 | fx), S1.y ^ (alwb1 | fx));
            if (COUNT)
                n_words += 4;
        }
        if (all_always || none_random)
            continue;
        if (COUNT && act)
            n_calls += 1;
        if (ha0)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w0, S0.x, R.x, m2a0);
        if (ha1)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w0 + 1u, S0.y, R.y, m2a1);
        if (hb0)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w1, S1.x, R.z, m2b0);
        if (hb1)
            q[atomicAdd(qn, 1)] = make_uint4((uint32_t)w1 + 1u, S1.y, R.w, m2b1);
        __syncwarp();
        int q_n = *qn;
        if (q_n >= 96) {  // full rounds, one queued word per lane, while 32 are queued
            do {
                q_n -= 32;
                const uint4 e = q[q_n + lane];
                unsigned int extra = 0;
                gtile_finish(jb, tb, e, upd, nb, Jx, Jy, Jz, gg, h, live0, live1, live2, always3,
                             T1x, T0, c1, c2m, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
            } while (q_n >= 32);
            if (lane == 0)
                *qn = q_n;
            __syncwarp();
        }
    }
    __syncthreads();
    const int n0q = s_qn[0], n1q = n0q + s_qn[1], n2q = n1q + s_qn[2], n3q = n2q + s_qn[3];
    for (int g = (int)threadIdx.x; g < n3q; g += kSweepThreads) {
        const int wq = g < n0q ? 0 : g < n1q ? 1 : g < n2q ? 2 : 3;
        const int off = g - (wq == 0 ? 0 : wq == 1 ? n0q : wq == 2 ? n1q : n2q);
        unsigned int extra = 0;
        gtile_finish(jb, tb, s_q[wq][off], upd, nb, Jx, Jy, Jz, gg, h, live0, live1, live2,
                     always3, T1x, T0, c1, c2m, c3, rk, extra);
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_calls + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// ---------------------------------------------------------------------------
// Heat bath, any side.  Per word-site one Philox call (stream 2, call 0, the
// word's own widx and replica): out0 is the coin word of class 3 (dE = 0, flip
// probability 1/2), and out1, out2, out3 hold the 16 leading bits of the first
// draws of the class pairs (2, 4), (1, 5), (0, 6), class u < 3 in the high
// half.  Call 128 + (2 - j) completes both first draws of the pair (j, 6 - j):
// (out0:out1) >> 16 and (out2:out3) >> 16.  Class u < 3 flips the lanes that
// the gaps of table C_u select; class u > 3 keeps the lanes that the gaps of
// C_(6-u) select and flips the rest (P(dE) + P(-dE) = 1).  Draw d >= 1 of
// class u is (out[2e] << 32) | out[2e + 1] of call 1 + u + 7 ((d - 1) div 2).
// Words whose leading bits might select a lane wait in a per-warp queue and
// are finished 32 at a time, as in the Metropolis kernels.
// ---------------------------------------------------------------------------
struct HeatPending {
    uint32_t w, sp, b0, b1, b2, c2;
};
constexpr int kHeatQueue = 64;  // entries per warp (at most 32 are added per step)

// Class masks u = 0..6 of a word from its bit-sliced count (u <= 6, so
// b2 & b1 & b0 never occurs).
struct HeatMasks {
    uint32_t M[7];
};

__device__ __forceinline__ HeatMasks heat_masks(uint32_t b2, uint32_t b1, uint32_t b0,
                                                uint32_t valid)
{
    const uint32_t lo = ~b2 & valid, hi = b2 & valid;
    HeatMasks m;
    m.M[0] = lo & ~(b1 | b0);
    m.M[1] = lo & ~b1 & b0;
    m.M[2] = lo & b1 & ~b0;
    m.M[3] = lo & b1 & b0;
    m.M[4] = hi & ~(b1 | b0);
    m.M[5] = hi & b0;
    m.M[6] = hi & b1;
    return m;
}

// Might the gaps select a lane of some class?  hl[j][n] = C_j[n] >> 48, or -1
// where no draw can select (n = 0, or class j without a table): a first draw
// whose 16 leading bits exceed it is >= C_j[n].
__device__ __forceinline__ bool heat_hit(const uint4 &R, const HeatMasks &m, const int (*hl)[33])
{
    bool h = (int)(R.y >> 16) <= hl[2][__popc(m.M[2])];
    h |= (int)(R.y & 0xFFFFu) <= hl[2][__popc(m.M[4])];
    h |= (int)(R.z >> 16) <= hl[1][__popc(m.M[1])];
    h |= (int)(R.z & 0xFFFFu) <= hl[1][__popc(m.M[5])];
    h |= (int)(R.w >> 16) <= hl[0][__popc(m.M[0])];
    h |= (int)(R.w & 0xFFFFu) <= hl[0][__popc(m.M[6])];
    return h;
}

// The flips of one word whose leading bits might select a lane: w its
// word-site, sp its spins, (b2 b1 b0) its class count, c2 its counter word.
__device__ __forceinline__ uint32_t heat_word_flips(const JobDev *__restrict__ jb, uint32_t w,
                                                    uint32_t b2, uint32_t b1, uint32_t b0,
                                                    uint32_t c2, uint32_t valid, uint32_t c1,
                                                    uint32_t c3, const uint32_t (&rk)[20],
                                                    const int (*hl)[33], unsigned int &calls)
{
    const uint4 R = dev::philox10_rk(make_uint4(w, c1, c2, c3), rk);
    ++calls;
    const HeatMasks m = heat_masks(b2, b1, b0, valid);
    uint32_t A = m.M[3] & R.x;
    const uint32_t lead[3] = {R.w, R.z, R.y};  // pair j = 0, 1, 2
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint32_t Ml = m.M[j], Mh = m.M[6 - j];
        const bool hit_l = (int)(lead[j] >> 16) <= hl[j][__popc(Ml)];
        const bool hit_h = (int)(lead[j] & 0xFFFFu) <= hl[j][__popc(Mh)];
        uint32_t keep = 0u;
        if (hit_l || hit_h) {
            const uint4 X =
                dev::philox10_rk(make_uint4(w, c1, c2 | (uint32_t)(128 + 2 - j), c3), rk);
            ++calls;
            if (hit_l)
                A |= gap_class<7>(jb, j, j, Ml,
                                  ((uint64_t)(lead[j] >> 16) << 48) |
                                      ((((uint64_t)X.x << 32) | X.y) >> 16),
                                  w, c1, c2, c3, rk, calls);
            if (hit_h)
                keep = gap_class<7>(jb, j, 6 - j, Mh,
                                    ((uint64_t)(lead[j] & 0xFFFFu) << 48) |
                                        ((((uint64_t)X.z << 32) | X.w) >> 16),
                                    w, c1, c2, c3, rk, calls);
        }
        A |= Mh & ~keep;
    }
    return A & valid;
}

__device__ __forceinline__ void heat_finish(const JobDev *__restrict__ jb, const HeatPending &e,
                                            uint32_t *__restrict__ upd, uint32_t valid,
                                            uint32_t c1, uint32_t c3, const uint32_t (&rk)[20],
                                            const int (*hl)[33], unsigned int &calls)
{
    upd[e.w] = e.sp ^ heat_word_flips(jb, e.w, e.b2, e.b1, e.b0, e.c2, valid, c1, c3, rk, hl,
                                      calls);
}

template <bool COUNT, int MAXJ>
__global__ void __launch_bounds__(kSweepThreads, 8)
    heat_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    __shared__ int s_hl[3][33];
    __shared__ HeatPending s_q[kSweepThreads / 32][kHeatQueue];
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33, g = i % 33;
        const bool live = ((J.meta >> u) & 1u) != 0 && g > 0;
        (&s_hl[0][0])[i] = live ? (int)((&jb->gC_hi[0][0])[i] >> 16) : -1;
    }
    __syncthreads();
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;  // this job has stopped (uniform over the block)

    const int h = P.h;
    const int lane = threadIdx.x & 31;
    HeatPending *q = s_q[threadIdx.x >> 5];
    int q_n = 0;  // warp-uniform queue length
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    const int cb = local - s * G.bps;
    const int n0 = G.n0, n1 = G.n1, n2 = G.n2;
    const bool fix_x = (G.fix & 1u) != 0;
    const bool fix_y = (G.fix & 2u) != 0;
    const uint32_t valid = G.valid;
    Axis az, ax, ay;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        az.sA[dir] = G.zsA[dir];
        az.sB[dir] = G.zsB[dir];
        az.mA[dir] = G.zmA[dir];
        az.mB[dir] = G.zmB[dir];
    }
    if (fix_x)
        load_axis(ax, jb->geo, 0);
    if (fix_y)
        load_axis(ay, jb->geo, 1);
    const uint32_t W = G.words;
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2h = dev::kStreamHeat | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    const int sz = n0 * n1;
    unsigned int n_words = 0, n_extra = 0;

    const int cols = G.cols;
    for (int k = 0; k < G.cpt; ++k) {
        const int col0 = (cb * G.cpt + k) * kSweepThreads + (int)threadIdx.x;
        const bool act = col0 < cols;  // lanes past the last column idle in step
        if (__all_sync(0xffffffffu, !act))
            break;
        const int col = act ? col0 : 0;
        const int y = (int)((__umulhi((uint32_t)col, G.magic) + (uint32_t)col) >> G.dshift);
        const int x = col - y * n0;
        int cxp = col + 1, cxm = col - 1, cyp = col + n0, cym = col - n0;
        const bool wxp = (x + 1 == n0), wxm = (x == 0), wyp = (y + 1 == n1), wym = (y == 0);
        if (wxp)
            cxp = col - (n0 - 1);
        if (wxm)
            cxm = col + (n0 - 1);
        if (wyp)
            cyp = col - (n1 - 1) * n0;
        if (wym)
            cym = col + (n1 - 1) * n0;
        // replica updated at word-site (x, y, z) in half-step h: h ^ ((x + y + z) & 1)
        const uint32_t c2e = c2h | ((uint32_t)(h ^ ((x + y) & 1)) << 11);  // even z
        uint32_t nz_prev = fixup(nb[col + (n2 - 1) * sz], az, 1);          // z' = -1
        uint32_t jz_prev = fixup(Jz[col + (n2 - 1) * sz], az, 1);          // bond below z' = 0
        uint32_t nz_cur = nb[col];
        for (int z = 0; z < n2; ++z) {
            const int w = col + z * sz;
            const uint32_t nz_next = (z + 1 < n2) ? nb[w + sz] : fixup(nb[col], az, 0);
            const uint32_t sp = upd[w];
            uint32_t nxp = nb[cxp + z * sz], nxm = nb[cxm + z * sz];
            uint32_t nyp = nb[cyp + z * sz], nym = nb[cym + z * sz];
            uint32_t jxm = Jx[cxm + z * sz], jym = Jy[cym + z * sz];
            if (fix_x) {
                if (wxp)
                    nxp = fixup(nxp, ax, 0);
                if (wxm) {
                    nxm = fixup(nxm, ax, 1);
                    jxm = fixup(jxm, ax, 1);
                }
            }
            if (fix_y) {
                if (wyp)
                    nyp = fixup(nyp, ay, 0);
                if (wym) {
                    nym = fixup(nym, ay, 1);
                    jym = fixup(jym, ay, 1);
                }
            }
            const uint32_t jz = Jz[w];
            const Count c = count6(sp ^ nxp ^ Jx[w], sp ^ nxm ^ jxm, sp ^ nyp ^ Jy[w],
                                   sp ^ nym ^ jym, sp ^ nz_next ^ jz, sp ^ nz_prev ^ jz_prev);
            nz_prev = nz_cur;
            nz_cur = nz_next;
            jz_prev = jz;

            const uint32_t c2 = c2e ^ ((uint32_t)(z & 1) << 11);
            const uint4 R = dev::philox10_rk(make_uint4((uint32_t)w, c1, c2, c3), rk);
            const HeatMasks m = heat_masks(c.b2, c.b1, c.b0, valid);
            const bool hit = act && heat_hit(R, m, s_hl);
            // no selection: class 3 by its coin, classes 4-6 flip whole
            if (act && !hit)
                upd[w] = sp ^ ((m.M[3] & R.x) | (c.b2 & valid));
            if (COUNT && act)
                ++n_words;
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                HeatPending &e = q[q_n + __popc(bal & ((1u << lane) - 1u))];
                e.w = (uint32_t)w;
                e.sp = sp;
                e.b0 = c.b0;
                e.b1 = c.b1;
                e.b2 = c.b2;
                e.c2 = c2;
            }
            q_n += __popc(bal);
            __syncwarp();
            if (q_n >= 32) {  // a full round: one queued word per lane
                q_n -= 32;
                const HeatPending e = q[q_n + lane];
                unsigned int extra = 0;
                heat_finish(jb, e, upd, valid, c1, c3, rk, s_hl, extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
            }
        }
    }
    if (lane < q_n) {  // the last, partial round
        const HeatPending e = q[lane];
        unsigned int extra = 0;
        heat_finish(jb, e, upd, valid, c1, c3, rk, s_hl, extra);
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_words + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// Heat bath for a table whose jobs all have side GL = 64 or 128, or (GL =
// kGeneralTile) the other sides of the general tile kernel, with the word
// lattice read at run time: the tiles of the Metropolis tile kernels (2 x 2
// word-sites times a segment of rows), one main call per word.  A queued word holds (word-site, spins before the
// update); its rare path counts its classes again from the neighbour area,
// which this half-step does not write, and draws its main call again.
template <int GL>
__device__ __forceinline__ void heat_tile_finish(const JobDev *__restrict__ jb, const uint4 &e,
                                                 uint32_t *__restrict__ upd,
                                                 const uint32_t *__restrict__ nb,
                                                 const uint32_t *__restrict__ Jx,
                                                 const uint32_t *__restrict__ Jy,
                                                 const uint32_t *__restrict__ Jz, int h,
                                                 uint32_t c1, uint32_t c2h, uint32_t c3,
                                                 const uint32_t (&rk)[20], const int (*hl)[33],
                                                 unsigned int &calls)
{
    constexpr int SLOG = GL == 128 ? 7 : 6;
    constexpr int N2 = GL / 32, SZ = GL * GL;
    const int w = (int)e.x;
    const uint32_t s = e.y;
    const int x = w & (GL - 1), y = (w >> SLOG) & (GL - 1), z = w >> (2 * SLOG);
    const uint32_t c2 = c2h | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
    const int wxp = x == GL - 1 ? w - (GL - 1) : w + 1;
    const int wxm = x == 0 ? w + (GL - 1) : w - 1;
    const int wyp = y == GL - 1 ? w - (GL - 1) * GL : w + GL;
    const int wym = y == 0 ? w + (GL - 1) * GL : w - GL;
    const int wzp = z == N2 - 1 ? w - (N2 - 1) * SZ : w + SZ;
    const int wzm = z == 0 ? w + (N2 - 1) * SZ : w - SZ;
    uint32_t nzp = nb[wzp], nzm = nb[wzm], jzm = Jz[wzm];
    if (z == N2 - 1)
        nzp = rot_zp(nzp);
    if (z == 0) {
        nzm = rot_zm(nzm);
        jzm = rot_zm(jzm);
    }
    const Count c = count6(s ^ nb[wxp] ^ Jx[w], s ^ nb[wxm] ^ Jx[wxm], s ^ nb[wyp] ^ Jy[w],
                           s ^ nb[wym] ^ Jy[wym], s ^ nzp ^ Jz[w], s ^ nzm ^ jzm);
    upd[w] = s ^ heat_word_flips(jb, (uint32_t)w, c.b2, c.b1, c.b0, c2, 0xffffffffu, c1, c3, rk,
                                 hl, calls);
}

// The rare path of a queued heat-bath word of a run-time lattice.
__device__ __forceinline__ void heat_gtile_finish(const JobDev *__restrict__ jb, const uint4 &e,
                                                  uint32_t *__restrict__ upd,
                                                  const uint32_t *__restrict__ nb,
                                                  const uint32_t *__restrict__ Jx,
                                                  const uint32_t *__restrict__ Jy,
                                                  const uint32_t *__restrict__ Jz,
                                                  const GTileGeo &gg, int h, uint32_t c1,
                                                  uint32_t c2h, uint32_t c3,
                                                  const uint32_t (&rk)[20], const int (*hl)[33],
                                                  unsigned int &calls)
{
    const int w = (int)e.x;
    const uint32_t s = e.y;
    const int x = w % gg.n0, r = w / gg.n0, y = r % gg.n1, z = r / gg.n1;
    const uint32_t c2 = c2h | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
    const Count c = gtile_count(w, s, x, y, z, nb, Jx, Jy, Jz, gg);
    upd[w] = s ^ heat_word_flips(jb, (uint32_t)w, c.b2, c.b1, c.b0, c2, 0xffffffffu, c1, c3, rk,
                                 hl, calls);
}

template <bool COUNT, int MAXJ, int GL, bool LOWT>
__global__ void __launch_bounds__(kSweepThreads, 7)
    heat_tile_kernel(const __grid_constant__ MetroParams<MAXJ> P, unsigned long long *counters)
{
    constexpr bool GEN = GL == kGeneralTile;  // the word lattice read at run time
    constexpr int N2 = GL / 32, SZ = GL * GL;
    constexpr int XP = GL / 2, ZP = N2 / 2;
    constexpr int XPLOG = GL == 128 ? 6 : 5;
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    __shared__ int s_hl[3][33];
    __shared__ uint4 s_q[kSweepThreads / 32][kTileQueue];
    __shared__ int s_qn[kSweepThreads / 32];
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33, g = i % 33;
        const bool live = ((J.meta >> u) & 1u) != 0 && g > 0;
        (&s_hl[0][0])[i] = live ? (int)((&jb->gC_hi[0][0])[i] >> 16) : -1;
    }
    if (threadIdx.x < kSweepThreads / 32)
        s_qn[threadIdx.x] = 0;
    __syncthreads();
    const int B1 = s_hl[1][32], B0 = s_hl[0][32];  // 32-lane bounds of the pairs (1, 5), (0, 6)
    const uint64_t t = jb->t + P.sweep_offset;
    if (t >= jb->t_end)
        return;

    const int h = P.h;
    const int lane = threadIdx.x & 31;
    uint4 *q = s_q[threadIdx.x >> 5];
    int *qn = &s_qn[threadIdx.x >> 5];
    const int Y = G.seg;
    const int local = (int)blockIdx.x - P.block_begin[j];
    const int s = local / G.bps;
    int tl = (local - s * G.bps) * kSweepThreads + (int)threadIdx.x;
    // lattice of words n0 x n1 x n2, compile-time for sides 64 and 128
    const int n0 = GEN ? G.n0 : GL, n1 = GEN ? G.n1 : GL, n2 = GEN ? G.n2 : N2;
    const int sz = n0 * n1;
    const uint32_t W = GEN ? G.words : (uint32_t)SZ * N2;
    GTileGeo gg;
    bool act = true;  // threads past the sample's last tile run on a valid tile, write nothing
    int x0, z0, y0;
    if constexpr (GEN) {
        gg.n0 = n0;
        gg.n1 = n1;
        gg.n2 = n2;
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            gg.ay.sA[dir] = G.ysA[dir];
            gg.ay.sB[dir] = G.ysB[dir];
            gg.ay.mA[dir] = G.ymA[dir];
            gg.ay.mB[dir] = G.ymB[dir];
            gg.az.sA[dir] = G.zsA[dir];
            gg.az.sB[dir] = G.zsB[dir];
            gg.az.mA[dir] = G.zmA[dir];
            gg.az.mB[dir] = G.zmB[dir];
        }
        const int xp = n0 >> 1, zp = n2 >> 1;
        act = tl < xp * zp * (n1 / Y);
        if (!act)
            tl = 0;
        x0 = 2 * (tl % xp);
        z0 = 2 * ((tl / xp) % zp);
        y0 = tl / xp / zp * Y;
    } else {
        // threads past the last segment of a row range run on a valid tile and
        // write nothing
        act = (tl >> XPLOG) / ZP * Y < G.row_n;
        if (!act)
            tl = 0;
        x0 = 2 * (tl & (XP - 1));
        z0 = 2 * ((tl >> XPLOG) & (ZP - 1));  // uniform over a warp (XP >= 32)
        y0 = G.row0 + (tl >> XPLOG) / ZP * Y;
    }
    uint32_t *__restrict__ upd = J.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = J.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = J.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2h = dev::kStreamHeat | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
    const int oz0 = z0 * sz, oz1 = oz0 + sz;
    const int ozm = (z0 == 0 ? n2 - 1 : z0 - 1) * sz;
    const int ozp = (z0 + 2 == n2 ? 0 : z0 + 2) * sz;
    const bool wrap_m = z0 == 0, wrap_p = z0 + 2 == n2;
    int xm, xq;
    if constexpr (GEN) {
        xm = x0 == 0 ? n0 - 1 : x0 - 1;
        xq = x0 + 2 == n0 ? 0 : x0 + 2;
    } else {
        xm = (x0 - 1) & (GL - 1);
        xq = (x0 + 2) & (GL - 1);
    }
    unsigned int n_words = 0, n_extra = 0;

    // the window; with a run-time lattice the row above a segment that starts
    // at y = 0 lies across the y wrap
    const int rym = GEN ? (y0 == 0 ? n1 - 1 : y0 - 1) * n0 : ((y0 - 1) & (GL - 1)) * GL;
    uint2 Nm0 = ld2(nb, x0 + rym + oz0), Nm1 = ld2(nb, x0 + rym + oz1);
    uint2 Jym0 = ld2(Jy, x0 + rym + oz0), Jym1 = ld2(Jy, x0 + rym + oz1);
    if (GEN && y0 == 0) {
        Nm0 = make_uint2(fixup(Nm0.x, gg.ay, 1), fixup(Nm0.y, gg.ay, 1));
        Nm1 = make_uint2(fixup(Nm1.x, gg.ay, 1), fixup(Nm1.y, gg.ay, 1));
        Jym0 = make_uint2(fixup(Jym0.x, gg.ay, 1), fixup(Jym0.y, gg.ay, 1));
        Jym1 = make_uint2(fixup(Jym1.x, gg.ay, 1), fixup(Jym1.y, gg.ay, 1));
    }
    uint2 Nc0 = ld2(nb, x0 + y0 * n0 + oz0), Nc1 = ld2(nb, x0 + y0 * n0 + oz1);
    for (int i = 0; i < Y; ++i) {
        const int y = y0 + i;
        const bool wrap_y = GEN && y + 1 == n1;  // only on a segment's last row
        const int ry = y * n0;
        const int ryp = GEN ? (wrap_y ? 0 : ry + n0) : ((y + 1) & (GL - 1)) * GL;
        const int w0 = x0 + ry + oz0, w1 = x0 + ry + oz1;  // the even-x words at z0, z0 + 1
        const uint2 S0 = ld2(upd, w0), S1 = ld2(upd, w1);
        uint2 Nn0 = ld2(nb, x0 + ryp + oz0), Nn1 = ld2(nb, x0 + ryp + oz1);
        if (wrap_y) {
            Nn0 = make_uint2(fixup(Nn0.x, gg.ay, 0), fixup(Nn0.y, gg.ay, 0));
            Nn1 = make_uint2(fixup(Nn1.x, gg.ay, 0), fixup(Nn1.y, gg.ay, 0));
        }
        uint2 Nzm = ld2(nb, x0 + ry + ozm), Nzp = ld2(nb, x0 + ry + ozp);
        uint2 Jzm = ld2(Jz, x0 + ry + ozm);
        const uint32_t Xm0 = nb[xm + ry + oz0], Xm1 = nb[xm + ry + oz1];
        const uint32_t Xp0 = nb[xq + ry + oz0], Xp1 = nb[xq + ry + oz1];
        const uint32_t Jxm0 = Jx[xm + ry + oz0], Jxm1 = Jx[xm + ry + oz1];
        const uint2 Jx0 = ld2(Jx, w0), Jx1 = ld2(Jx, w1);
        const uint2 Jy0 = ld2(Jy, w0), Jy1 = ld2(Jy, w1);
        const uint2 Jz0 = ld2(Jz, w0), Jz1 = ld2(Jz, w1);
        if constexpr (GEN) {
            if (wrap_m) {
                Nzm = make_uint2(fixup(Nzm.x, gg.az, 1), fixup(Nzm.y, gg.az, 1));
                Jzm = make_uint2(fixup(Jzm.x, gg.az, 1), fixup(Jzm.y, gg.az, 1));
            }
            if (wrap_p)
                Nzp = make_uint2(fixup(Nzp.x, gg.az, 0), fixup(Nzp.y, gg.az, 0));
        } else {
            if (wrap_m) {
                Nzm = make_uint2(rot_zm(Nzm.x), rot_zm(Nzm.y));
                Jzm = make_uint2(rot_zm(Jzm.x), rot_zm(Jzm.y));
            }
            if (wrap_p)
                Nzp = make_uint2(rot_zp(Nzp.x), rot_zp(Nzp.y));
        }
        // replica of word (x0, y, z0); the other three alternate with x and z
        const uint32_t c2a = c2h | ((uint32_t)(h ^ (y & 1)) << 11);
        const uint32_t c2b = c2a ^ (1u << 11);
        // words a0 = (x0, z0), a1 = (x0 + 1, z0), b0 = (x0, z0 + 1), b1 = (x0 + 1, z0 + 1)
        const uint32_t wd[4] = {(uint32_t)w0, (uint32_t)w0 + 1u, (uint32_t)w1, (uint32_t)w1 + 1u};
        const uint32_t sp[4] = {S0.x, S0.y, S1.x, S1.y};
        const uint32_t c2w[4] = {c2a, c2b, c2b, c2a};
        // the six bond inputs of each word (x neighbours inside the pair come
        // from the other word of the pair, z neighbours from the other z row)
        const uint32_t in[4][6] = {
            {Nc0.y ^ Jx0.x, Xm0 ^ Jxm0, Nn0.x ^ Jy0.x, Nm0.x ^ Jym0.x, Nc1.x ^ Jz0.x,
             Nzm.x ^ Jzm.x},
            {Xp0 ^ Jx0.y, Nc0.x ^ Jx0.x, Nn0.y ^ Jy0.y, Nm0.y ^ Jym0.y, Nc1.y ^ Jz0.y,
             Nzm.y ^ Jzm.y},
            {Nc1.y ^ Jx1.x, Xm1 ^ Jxm1, Nn1.x ^ Jy1.x, Nm1.x ^ Jym1.x, Nzp.x ^ Jz1.x,
             Nc0.x ^ Jz0.x},
            {Xp1 ^ Jx1.y, Nc1.x ^ Jx1.x, Nn1.y ^ Jy1.y, Nm1.y ^ Jym1.y, Nzp.y ^ Jz1.y,
             Nc0.y ^ Jz0.y}};
        Nm0 = Nc0;
        Nm1 = Nc1;
        Nc0 = Nn0;
        Nc1 = Nn1;
        Jym0 = Jy0;
        Jym1 = Jy1;
        uint32_t out[4];
        bool hit[4];
        // the four words' main calls advance round by round together: each
        // round key serves four calls and the four multiply chains overlap
        uint4 RR[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            RR[k] = make_uint4(wd[k], c1, c2w[k], c3);
        dev::philox10_rk_x4(RR, rk);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t v = sp[k];
            const Count c = count6(v ^ in[k][0], v ^ in[k][1], v ^ in[k][2], v ^ in[k][3],
                                   v ^ in[k][4], v ^ in[k][5]);
            const uint4 R = RR[k];
            uint32_t m3;
            if (LOWT) {
                // the pairs (1, 5) and (0, 6) against their 32-lane bounds: a superset
                // of the per-count test that needs neither their masks nor popcounts
                const uint32_t lo = ~c.b2;
                const uint32_t m2 = lo & c.b1 & ~c.b0, m4 = c.b2 & ~(c.b1 | c.b0);
                m3 = lo & c.b1 & c.b0;
                bool h = (int)(R.y >> 16) <= s_hl[2][__popc(m2)];
                h |= (int)(R.y & 0xFFFFu) <= s_hl[2][__popc(m4)];
                h |= (int)(R.z >> 16) <= B1;
                h |= (int)(R.z & 0xFFFFu) <= B1;
                h |= (int)(R.w >> 16) <= B0;
                h |= (int)(R.w & 0xFFFFu) <= B0;
                hit[k] = h;
            } else {
                const HeatMasks m = heat_masks(c.b2, c.b1, c.b0, 0xffffffffu);
                hit[k] = heat_hit(R, m, s_hl);
                m3 = m.M[3];
            }
            // without a selection: class 3 by its coin, classes 4-6 flip whole
            out[k] = v ^ ((m3 & R.x) | c.b2);
        }
        // every word is written; a queued word is written again by the rare path
        if (act) {
            *reinterpret_cast<uint2 *>(upd + w0) = make_uint2(out[0], out[1]);
            *reinterpret_cast<uint2 *>(upd + w1) = make_uint2(out[2], out[3]);
            if (COUNT)
                n_words += 4;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (act && hit[k])
                q[atomicAdd(qn, 1)] = make_uint4(wd[k], sp[k], 0u, 0u);
        __syncwarp();
        int q_n = *qn;
        if (q_n >= 96) {  // full rounds, one queued word per lane, while 32 are queued
            do {
                q_n -= 32;
                const uint4 e = q[q_n + lane];
                unsigned int extra = 0;
                if constexpr (GEN)
                    heat_gtile_finish(jb, e, upd, nb, Jx, Jy, Jz, gg, h, c1, c2h, c3, rk, s_hl,
                                      extra);
                else
                    heat_tile_finish<GL>(jb, e, upd, nb, Jx, Jy, Jz, h, c1, c2h, c3, rk, s_hl,
                                         extra);
                if (COUNT)
                    n_extra += extra;
                __syncwarp();
            } while (q_n >= 32);
            if (lane == 0)
                *qn = q_n;
            __syncwarp();
        }
    }
    // the words still queued in the block's four warps, pooled
    __syncthreads();
    const int n0q = s_qn[0], n1q = n0q + s_qn[1], n2q = n1q + s_qn[2], n3q = n2q + s_qn[3];
    for (int g = (int)threadIdx.x; g < n3q; g += kSweepThreads) {
        const int wq = g < n0q ? 0 : g < n1q ? 1 : g < n2q ? 2 : 3;
        const int off = g - (wq == 0 ? 0 : wq == 1 ? n0q : wq == 2 ? n1q : n2q);
        unsigned int extra = 0;
        if constexpr (GEN)
            heat_gtile_finish(jb, s_q[wq][off], upd, nb, Jx, Jy, Jz, gg, h, c1, c2h, c3, rk,
                              s_hl, extra);
        else
            heat_tile_finish<GL>(jb, s_q[wq][off], upd, nb, Jx, Jy, Jz, h, c1, c2h, c3, rk,
                                 s_hl, extra);
        if (COUNT)
            n_extra += extra;
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_words + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

// ---------------------------------------------------------------------------
// Metropolis sweeps with the whole sample resident in shared memory: one block
// per sample loads both areas and the three coupling arrays once, runs every
// sweep of the launch (both half-steps, __syncthreads between them) out of
// shared memory and writes the spins back at the end.  For samples small
// enough to fit (side <= 64), where one sample is too little work to fill
// the GPU for a single half-step, so that per-half-step launches would run at
// launch latency.  Any side: the word lattice n0 x n1 x n2 and the lane
// realignment at the wraps come from the geometry, as in metro_kernel.
//   pass 1: a thread takes a quad of word-sites (x' even, x' + 1) x (z' even,
//     z' + 1) at one y', draws the quad's main call, and writes each word
//     with its outright flips unless the leading bits of its first draws might
//     select a lane; such words go to a block queue (word-site, main bits);
//   pass 2: the queued words are counted again from the neighbour area, which
//     this half-step does not write, and finished exactly (finish_word).
// The draws are those of every other Metropolis kernel, so a job's results do
// not depend on the kernel that runs it.
// ---------------------------------------------------------------------------
// 512 threads: half the work between the barriers of a half-step, and twice
// the warps to cover shared-memory latency, against 256 (sides 48 and 64 run
// 17-28% faster, side 32 the same).
constexpr int kResThreads = 512;

// The lane realignment of the resident kernel: z (every side: a z wrap of a
// side with one word along z is every word's) in registers, x and y (only the
// sides below 32 and those whose y wrap realigns) from shared memory.
struct ResGeo {
    int n0, n1, n2, sz;
    bool fix_x, fix_y;
    Axis az;
    const Axis *axy;  // x, y
};

__device__ __forceinline__ uint32_t res_fix_x(uint32_t w, const ResGeo &g, int dir)
{
    return fixup(w, g.axy[0], dir);
}

__device__ __forceinline__ uint32_t res_fix_y(uint32_t w, const ResGeo &g, int dir)
{
    return fixup(w, g.axy[1], dir);
}

__device__ __forceinline__ uint32_t res_fix_z(uint32_t w, const ResGeo &g, int dir)
{
    return fixup(w, g.az, dir);
}

// The bit-sliced count of the word at word-site w = (x, y, z) with spins s,
// its neighbours in area nb and its bonds in Jx, Jy, Jz (all in shared memory).
__device__ __forceinline__ Count res_count(const uint32_t *nb, const uint32_t *Jx,
                                           const uint32_t *Jy, const uint32_t *Jz, uint32_t s,
                                           int x, int y, int z, int w, const ResGeo &g)
{
    const bool exp_ = x + 1 == g.n0, exm = x == 0, eyp = y + 1 == g.n1, eym = y == 0;
    const bool ezp = z + 1 == g.n2, ezm = z == 0;
    const int wxp = exp_ ? w - (g.n0 - 1) : w + 1;
    const int wxm = exm ? w + (g.n0 - 1) : w - 1;
    const int wyp = eyp ? w - (g.n1 - 1) * g.n0 : w + g.n0;
    const int wym = eym ? w + (g.n1 - 1) * g.n0 : w - g.n0;
    const int wzp = ezp ? w - (g.n2 - 1) * g.sz : w + g.sz;
    const int wzm = ezm ? w + (g.n2 - 1) * g.sz : w - g.sz;
    uint32_t nxp = nb[wxp], nxm = nb[wxm], jxm = Jx[wxm];
    uint32_t nyp = nb[wyp], nym = nb[wym], jym = Jy[wym];
    uint32_t nzp = nb[wzp], nzm = nb[wzm], jzm = Jz[wzm];
    if (g.fix_x) {
        if (exp_)
            nxp = res_fix_x(nxp, g, 0);
        if (exm) {
            nxm = res_fix_x(nxm, g, 1);
            jxm = res_fix_x(jxm, g, 1);
        }
    }
    if (g.fix_y) {
        if (eyp)
            nyp = res_fix_y(nyp, g, 0);
        if (eym) {
            nym = res_fix_y(nym, g, 1);
            jym = res_fix_y(jym, g, 1);
        }
    }
    if (ezp)
        nzp = res_fix_z(nzp, g, 0);
    if (ezm) {
        nzm = res_fix_z(nzm, g, 1);
        jzm = res_fix_z(jzm, g, 1);
    }
    return count6(s ^ nxp ^ Jx[w], s ^ nxm ^ jxm, s ^ nyp ^ Jy[w], s ^ nym ^ jym, s ^ nzp ^ Jz[w],
                  s ^ nzm ^ jzm);
}

// Dynamic shared memory of a resident block for a sample of W words per area:
// areas 0 and 1, Jx, Jy, Jz, and the queue of up to W (word-site, main bits).
__host__ __device__ constexpr size_t res_smem_bytes(int W)
{
    return (size_t)W * (5 * sizeof(uint32_t) + sizeof(uint2));
}

template <bool COUNT, int MAXJ>
__global__ void __launch_bounds__(kResThreads, 1)
    metro_res_kernel(const __grid_constant__ MetroParams<MAXJ> P, uint32_t n_sweeps,
                     unsigned long long *counters)
{
    int j = 0;
    {
        int lo = 0, hi = P.n_jobs - 1;
        const int b = (int)blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.block_begin[mid] <= b)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    const MetroJob &J = P.job[j];
    const MetroGeo &G = P.geo[(J.meta >> 8) & 0xFFu];
    const JobDev *__restrict__ jb = P.jobs_dev + j;
    uint32_t rk[20];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    extern __shared__ __align__(16) uint32_t res_smem[];
    __shared__ uint32_t s_gh[3][33];
    __shared__ int s_qn;
    const int W = (int)G.words;
    uint32_t *const sJx = res_smem + 2 * W;
    uint32_t *const sJy = sJx + W;
    uint32_t *const sJz = sJy + W;
    uint2 *const queue = reinterpret_cast<uint2 *>(res_smem + 5 * W);
    for (int i = threadIdx.x; i < 3 * 33; i += blockDim.x) {
        const int u = i / 33;
        const uint32_t hi = (&jb->gC_hi[0][0])[i];
        (&s_gh[0][0])[i] = u == 2 ? lead2(hi) : u == 1 ? lead1(hi) : lead0(hi);
    }
    const int s = (int)blockIdx.x - P.block_begin[j];
    uint32_t *__restrict__ gsp = J.spins + (size_t)s * 2 * W;
    const uint32_t *__restrict__ gJ = J.J + (size_t)s * 3 * W;
    // W is a multiple of 8 (every side of the word lattice is even)
    for (int i = threadIdx.x; i < W / 2; i += blockDim.x) {
        reinterpret_cast<uint4 *>(res_smem)[i] = reinterpret_cast<const uint4 *>(gsp)[i];
        if (i < 3 * W / 4)
            reinterpret_cast<uint4 *>(sJx)[i] = reinterpret_cast<const uint4 *>(gJ)[i];
    }
    for (int i = W / 2 + threadIdx.x; i < 3 * W / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(sJx)[i] = reinterpret_cast<const uint4 *>(gJ)[i];
    __shared__ Axis s_axy[2];
    if (threadIdx.x == 0) {
        s_qn = 0;
        if (G.fix & 1u)
            load_axis(s_axy[0], jb->geo, 0);
        if (G.fix & 2u)
            load_axis(s_axy[1], jb->geo, 1);
    }
    __syncthreads();

    ResGeo g;
    g.n0 = G.n0;
    g.n1 = G.n1;
    g.n2 = G.n2;
    g.sz = G.n0 * G.n1;
    g.fix_x = (G.fix & 1u) != 0;
    g.fix_y = (G.fix & 2u) != 0;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        g.az.sA[dir] = G.zsA[dir];
        g.az.sB[dir] = G.zsB[dir];
        g.az.mA[dir] = G.zmA[dir];
        g.az.mB[dir] = G.zmB[dir];
    }
    g.axy = s_axy;
    const uint32_t valid = G.valid;
    const bool all_always = (J.meta >> 3) & 1u, none_random = (J.meta >> 4) & 1u;
    const uint32_t live0 = 0u - (J.meta & 1u), live1 = 0u - ((J.meta >> 1) & 1u),
                   live2 = 0u - ((J.meta >> 2) & 1u);
    const uint32_t c3 = ((uint32_t)s + (J.meta >> 16)) / J.rng_group;
    const int hx = g.n0 >> 1, quads = hx * g.n1 * (g.n2 >> 1);
    unsigned int n_words = 0, n_calls = 0, n_extra = 0;

    for (uint32_t k = 0; k < n_sweeps; ++k) {
        const uint64_t t = jb->t + P.sweep_offset + k;
        if (t >= jb->t_end)
            break;  // the job stops here (uniform over the block)
        const uint32_t c1 = (uint32_t)t;
        const uint32_t c2m = dev::kStreamMetropolis | (((uint32_t)(t >> 32) & 0xFFFFu) << 12);
        for (int h = 0; h < 2; ++h) {
            uint32_t *const upd = h ? res_smem + W : res_smem;
            const uint32_t *const nb = h ? res_smem : res_smem + W;
            for (int qd = threadIdx.x; qd < quads; qd += kResThreads) {
                const int xq = qd % hx, r = qd / hx;
                const int y = r % g.n1, z0 = (r / g.n1) * 2, x0 = 2 * xq;
                const int w0 = x0 + g.n0 * y + g.sz * z0;
                const int ws[4] = {w0, w0 + 1, w0 + g.sz, w0 + g.sz + 1};
                uint32_t sp[4], alw[4];
                Classes kc[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    sp[q] = upd[ws[q]];
                    const Count c = res_count(nb, sJx, sJy, sJz, sp[q], x0 + (q & 1), y,
                                              z0 + (q >> 1), ws[q], g);
                    alw[q] = c.b2 | (c.b1 & c.b0);
                    kc[q] = classes(c, alw[q], valid, live0, live1, live2);
                }
                if (COUNT)
                    n_words += 4;
                if (all_always || none_random) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        upd[ws[q]] = sp[q] ^ ((all_always ? 0xffffffffu : alw[q]) & valid);
                    continue;
                }
                // the quad's main call: its first word-site, the replica there
                const uint32_t c2q = c2m | ((uint32_t)(h ^ (y & 1)) << 11);
                const uint4 R = dev::philox10_rk(make_uint4((uint32_t)w0, c1, c2q, c3), rk);
                if (COUNT)
                    n_calls += 1;
                const uint32_t M[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (class_hit(kc[q], M[q], s_gh))
                        queue[atomicAdd(&s_qn, 1)] = make_uint2((uint32_t)ws[q], M[q]);
                    else
                        upd[ws[q]] = sp[q] ^ (alw[q] & valid);
                }
            }
            __syncthreads();
            const int nq = s_qn;
            for (int i = threadIdx.x; i < nq; i += kResThreads) {
                const uint2 e = queue[i];
                const int w = (int)e.x;
                const int x = w % g.n0, r = w / g.n0, y = r % g.n1, z = r / g.n1;
                const uint32_t sw = upd[w];  // not written in pass 1
                const Count c = res_count(nb, sJx, sJy, sJz, sw, x, y, z, w, g);
                const uint32_t a = c.b2 | (c.b1 & c.b0);
                const Classes kc = classes(c, a, valid, live0, live1, live2);
                Pending p;
                p.w = (uint32_t)w;
                p.base = sw ^ (a & valid);
                p.M0 = kc.M0;
                p.M1 = kc.M1;
                p.M2 = kc.M2;
                p.c2 = c2m | ((uint32_t)(h ^ ((x + y + z) & 1)) << 11);
                p.lead = e.y;
                unsigned int extra = 0;
                finish_word(jb, p, upd, valid, c1, c3, rk, extra);
                if (COUNT)
                    n_extra += extra;
            }
            __syncthreads();
            if (threadIdx.x == 0)
                s_qn = 0;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < W / 2; i += blockDim.x)
        reinterpret_cast<uint4 *>(gsp)[i] = reinterpret_cast<const uint4 *>(res_smem)[i];
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)n_words);
        atomicAdd(&counters[1], (unsigned long long)(n_calls + n_extra));
        atomicAdd(&counters[2], (unsigned long long)n_extra);
    }
}

__global__ void advance_time_kernel(JobDev *jobs, int n_jobs, uint64_t n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_jobs) {
        const uint64_t t = jobs[j].t + n;
        jobs[j].t = t < jobs[j].t_end ? t : jobs[j].t_end;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void fill_job_keys(JobDev *jd, uint64_t seed)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        jd->rk[2 * r] = k0;
        jd->rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

void fill_job_thresholds(JobDev *jd, const Thr &thr)
{
    for (int u = 0; u < 3; ++u)
        for (int g = 0; g < 33; ++g) {
            jd->gC_hi[u][g] = (uint32_t)(thr.geoC[u][g] >> 32);
            jd->gC_lo[u][g] = (uint32_t)thr.geoC[u][g];
        }
    jd->geo_live = thr.geo_live;
    jd->always_u = thr.always_u;
    jd->rule = thr.rule;
    jd->all_always = thr.all_always;
    jd->none_random = thr.none_random;
}

void fill_job_layout(JobDev *jd, int cols_per_thread)
{
    const Geo &g = jd->geo;
    jd->cols = g.n[0] * g.n[1];
    // q = (umulhi(c, m) + c) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1;
    // exact for c + umulhi(c, m) < 2^32 (here c < 2^21)
    const uint32_t d = (uint32_t)g.n[0];
    int l = 0;
    while ((1u << l) < d)
        ++l;
    const uint64_t m = (((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1;
    jd->div_n0_magic = (uint32_t)m;
    jd->div_n0_shift = l;
    jd->cols_per_thread = cols_per_thread < 1 ? 1 : cols_per_thread;
    const int per_block = kSweepThreads * jd->cols_per_thread;
    jd->blocks_per_sample = (jd->cols + per_block - 1) / per_block;
}

// the bounded waits of the staged kernel (set_wait_policy)
static std::atomic<uint32_t> g_wait_limit{1u << 22};
static std::atomic<uint32_t> g_wait_mode{0u};

static void metro_geo(MetroGeo &g, const JobDev &jd)
{
    std::memset(&g, 0, sizeof(g));
    g.n0 = jd.geo.n[0];
    g.n1 = jd.geo.n[1];
    g.n2 = jd.geo.n[2];
    g.cols = jd.cols;
    g.bps = jd.blocks_per_sample;
    g.cpt = jd.cols_per_thread;
    g.words = (uint32_t)jd.geo.words;
    g.valid = jd.geo.valid;
    g.magic = jd.div_n0_magic;
    g.dshift = jd.div_n0_shift;
    g.fix = (jd.geo.k[0] > 1 ? 1u : 0u) | (jd.geo.k[1] > 1 ? 2u : 0u);
    for (int dir = 0; dir < 2; ++dir) {
        g.zsA[dir] = jd.geo.sA[2][dir];
        g.zsB[dir] = jd.geo.sB[2][dir];
        g.zmA[dir] = jd.geo.mA[2][dir];
        g.zmB[dir] = jd.geo.mB[2][dir];
        g.ysA[dir] = jd.geo.sA[1][dir];
        g.ysB[dir] = jd.geo.sB[1][dir];
        g.ymA[dir] = jd.geo.mA[1][dir];
        g.ymB[dir] = jd.geo.mB[1][dir];
    }
}

static void metro_job(MetroJob &m, const JobDev &jd, int geo_index)
{
    m.spins = jd.spins;
    m.J = jd.J;
    m.key0 = jd.rk[0];
    m.key1 = jd.rk[1];
    m.rng_group = jd.rng_group;
    m.meta = (jd.geo_live & 7u) | (jd.all_always ? 8u : 0u) | (jd.none_random ? 16u : 0u) |
             ((uint32_t)geo_index << 8) | ((uint32_t)jd.first_sample << 16);
}

// Tiles (2 x 2 word-sites of one row) of all tile-kernel runs that
// launch_sweep_table spreads over streams at once, 0 outside such a set.
static thread_local long t_tiles_shared = 0;

// Jobs host[0..cnt) in one launch sequence; all of them share at most
// kMetroMaxGeo (side, layout) geometries.
template <int MAXJ, int GL, bool HEAT = false>
static void launch_metro_chunk(const JobDev *host, const JobDev *dev, int cnt, uint64_t n,
                               cudaStream_t stream, unsigned long long *counters, int half)
{
    MetroParams<MAXJ> p;
    std::memset(p.geo, 0, sizeof(p.geo));
    p.jobs_dev = dev;
    p.n_jobs = cnt;
    p.block_begin[0] = 0;
    p.wait_limit = g_wait_limit;
    p.wait_mode = g_wait_mode;
    int n_geo = 0;
    int geo_L[kMetroMaxGeo], geo_cpt[kMetroMaxGeo], geo_lo[kMetroMaxGeo], geo_hi[kMetroMaxGeo];
    // the rows a job's tile launch updates: all, or its row range (sides 64, 128)
    auto rows_of = [](const JobDev &jd) {
        return (GL == 64 || GL == 128) ? jd.row_hi - jd.row_lo : jd.geo.n[1];
    };
    // tile kernels: rows per thread from the launch shape, halved (down to 2)
    // while the launch would hold fewer than four blocks per SM.  Runs that
    // share the GPU on streams count the tiles of all of them (t_tiles_shared):
    // the GPU is full as long as the set is, so a small run of the set need not
    // take shorter rows
    int y_max = 16;
    if (GL != 0) {
        long tiles = 0;  // tiles of one row, 2 x 2 word-sites each
        for (int i = 0; i < cnt; ++i)
            tiles += (long)host[i].n_samples * (host[i].geo.n[0] / 2) * (host[i].geo.n[2] / 2) *
                     rows_of(host[i]);
        tiles = std::max(tiles, t_tiles_shared);
        while (y_max > 2 && tiles / y_max / kSweepThreads < 4L * kTileMinSMs)
            y_max >>= 1;
        // a launch that would not even give every SM a block takes single rows:
        // the lone samples of a serving tail run at the latency of short rows
        if (y_max == 2 && tiles / 2 / kSweepThreads < kTileMinSMs)
            y_max = 1;
    }
    for (int i = 0; i < cnt; ++i) {
        const JobDev &jd = host[i];
        int gi = 0;
        const bool ranged = GL == 64 || GL == 128;
        while (gi < n_geo &&
               !(geo_L[gi] == jd.geo.L && geo_cpt[gi] == jd.cols_per_thread &&
                 (!ranged || (geo_lo[gi] == jd.row_lo && geo_hi[gi] == jd.row_hi))))
            ++gi;
        if (gi == n_geo) {
            geo_L[gi] = jd.geo.L;
            geo_cpt[gi] = jd.cols_per_thread;
            geo_lo[gi] = jd.row_lo;
            geo_hi[gi] = jd.row_hi;
            metro_geo(p.geo[gi], jd);
            if (GL != 0) {
                // tiles of 2 x 2 word-sites times a segment of Y = 4, 8 or 16 rows
                // (fewer where the row count of the word lattice, or of the job's
                // row range, needs it)
                const int n_rows = rows_of(jd);
                int Y = std::min(y_max,
                                 jd.cols_per_thread >= 4 ? 16 : jd.cols_per_thread >= 2 ? 8 : 4);
                while (n_rows % Y != 0)
                    Y >>= 1;
                const int threads = (jd.geo.n[0] / 2) * (jd.geo.n[2] / 2) * (n_rows / Y);
                p.geo[gi].seg = Y;
                p.geo[gi].row0 = ranged ? jd.row_lo : 0;
                p.geo[gi].row_n = n_rows;
                p.geo[gi].bps = (threads + kSweepThreads - 1) / kSweepThreads;
            }
            ++n_geo;
        }
        metro_job(p.job[i], jd, gi);
        p.block_begin[i + 1] = p.block_begin[i] + jd.n_samples * p.geo[gi].bps;
    }
    const int grid = p.block_begin[cnt];
    if (grid == 0)
        return;
    // the classes dE = 8 and 12 take the 32-lane bound test when their tables
    // are small for every job (C_u[32] < 2^56) and no class is accepted outright
    bool lowt = true;
    for (int i = 0; i < cnt; ++i)
        lowt = lowt && (host[i].gC_hi[1][32] >> 24) == 0u && (host[i].gC_hi[0][32] >> 24) == 0u &&
               (host[i].always_u & 7u) == 0u;
    for (uint64_t k = 0; k < n; ++k)
        for (int h = 0; h < 2; ++h) {
            if (half >= 0 && h != half)
                continue;
            p.h = h;
            p.sweep_offset = (uint32_t)k;
            if constexpr (HEAT && GL != 0) {
                if (counters) {
                    if (lowt)
                        heat_tile_kernel<true, MAXJ, GL, true>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                    else
                        heat_tile_kernel<true, MAXJ, GL, false>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                } else if (lowt) {
                    heat_tile_kernel<false, MAXJ, GL, true>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                } else {
                    heat_tile_kernel<false, MAXJ, GL, false>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                }
            } else if constexpr (HEAT) {
                if (counters)
                    heat_kernel<true, MAXJ><<<grid, kSweepThreads, 0, stream>>>(p, counters);
                else
                    heat_kernel<false, MAXJ><<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
            } else if constexpr (GL == kGeneralTile) {
                if (counters) {
                    if (lowt)
                        metro_gtile_kernel<true, MAXJ, true>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                    else
                        metro_gtile_kernel<true, MAXJ, false>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                } else if (lowt) {
                    metro_gtile_kernel<false, MAXJ, true>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                } else {
                    metro_gtile_kernel<false, MAXJ, false>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                }
            } else if constexpr (GL == 128) {
                const bool staged = lowt && (host[0].variant & 1);
                if (staged) {
                    if (counters)
                        metro_stage_kernel<true, MAXJ>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                    else
                        metro_stage_kernel<false, MAXJ>
                            <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                } else if (counters) {
                    if (lowt)
                        metro_tile_kernel<true, MAXJ, GL, true>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                    else
                        metro_tile_kernel<true, MAXJ, GL, false>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                } else if (lowt) {
                    metro_tile_kernel<false, MAXJ, GL, true>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                } else {
                    metro_tile_kernel<false, MAXJ, GL, false>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                }
            } else if constexpr (GL != 0) {
                if (counters) {
                    if (lowt)
                        metro_tile_kernel<true, MAXJ, GL, true>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                    else
                        metro_tile_kernel<true, MAXJ, GL, false>
                            <<<grid, kSweepThreads, 0, stream>>>(p, counters);
                } else if (lowt) {
                    metro_tile_kernel<false, MAXJ, GL, true>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                } else {
                    metro_tile_kernel<false, MAXJ, GL, false>
                        <<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
                }
            } else {
                if (counters)
                    metro_kernel<true, MAXJ><<<grid, kSweepThreads, 0, stream>>>(p, counters);
                else
                    metro_kernel<false, MAXJ><<<grid, kSweepThreads, 0, stream>>>(p, nullptr);
            }
            count_launches(1);
        }
}

// The sample-resident kernel over jobs host[0..cnt): one block per sample, up
// to kResSweepsPerLaunch sweeps per launch.
template <bool COUNT, int MAXJ>
static void res_launch(const MetroParams<MAXJ> &p, int grid, size_t smem, uint32_t sweeps,
                       cudaStream_t stream, unsigned long long *counters)
{
    metro_res_kernel<COUNT, MAXJ><<<grid, kResThreads, smem, stream>>>(p, sweeps, counters);
    count_launches(1);
}

template <bool COUNT, int MAXJ>
static cudaError_t res_opt_in()
{
    return cudaFuncSetAttribute(metro_res_kernel<COUNT, MAXJ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)res_smem_bytes(kResMaxL * kResMaxL * kResMaxL / 32));
}

template <int MAXJ>
static void launch_res_chunk(const JobDev *host, const JobDev *dev, int cnt, uint64_t n,
                             cudaStream_t stream, unsigned long long *counters)
{
    MetroParams<MAXJ> p;
    std::memset(p.geo, 0, sizeof(p.geo));
    p.jobs_dev = dev;
    p.n_jobs = cnt;
    p.h = 0;
    p.wait_limit = g_wait_limit;
    p.wait_mode = g_wait_mode;
    p.block_begin[0] = 0;
    int n_geo = 0, geo_L[kMetroMaxGeo], W_max = 0;
    for (int i = 0; i < cnt; ++i) {
        const JobDev &jd = host[i];
        int gi = 0;
        while (gi < n_geo && geo_L[gi] != jd.geo.L)
            ++gi;
        if (gi == n_geo) {
            geo_L[gi] = jd.geo.L;
            metro_geo(p.geo[gi], jd);
            p.geo[gi].bps = 1;
            ++n_geo;
        }
        metro_job(p.job[i], jd, gi);
        p.block_begin[i + 1] = p.block_begin[i] + jd.n_samples;
        W_max = std::max(W_max, jd.geo.words);
    }
    const int grid = p.block_begin[cnt];
    if (grid == 0)
        return;
    const size_t smem = res_smem_bytes(W_max);
    for (uint64_t done = 0; done < n; done += kResSweepsPerLaunch) {
        p.sweep_offset = (uint32_t)done;
        const uint32_t k = (uint32_t)std::min<uint64_t>(kResSweepsPerLaunch, n - done);
        if (counters)
            res_launch<true, MAXJ>(p, grid, smem, k, stream, counters);
        else
            res_launch<false, MAXJ>(p, grid, smem, k, stream, nullptr);
    }
}

// Jobs host[0..cnt) of one run of the Metropolis table: side GLR (64 or 128,
// the tile kernel) or any sides (GLR = 0, the column kernel), in chunks of at
// most kMetroMaxJobs jobs and kMetroMaxGeo geometries per launch.
template <bool HEAT = false>
static void launch_metro_run(const JobDev *host, const JobDev *dev, int cnt, int GLR, uint64_t n,
                             cudaStream_t stream, unsigned long long *counters, int half)
{
    for (int first = 0, c = 0; first < cnt; first += c) {
        int n_geo = 0, geo_L[kMetroMaxGeo], geo_cpt[kMetroMaxGeo], geo_lo[kMetroMaxGeo],
            geo_hi[kMetroMaxGeo];
        for (c = 0; first + c < cnt && c < kMetroMaxJobs; ++c) {
            const JobDev &jd = host[first + c];
            int gi = 0;
            while (gi < n_geo &&
                   !(geo_L[gi] == jd.geo.L && geo_cpt[gi] == jd.cols_per_thread &&
                     geo_lo[gi] == jd.row_lo && geo_hi[gi] == jd.row_hi))
                ++gi;
            if (gi == n_geo) {
                if (n_geo == kMetroMaxGeo)
                    break;
                geo_L[gi] = jd.geo.L;
                geo_cpt[gi] = jd.cols_per_thread;
                geo_lo[gi] = jd.row_lo;
                geo_hi[gi] = jd.row_hi;
                ++n_geo;
            }
        }
        const JobDev *h = host + first;
        const JobDev *d = dev + first;
        if (!HEAT && GLR == kResidentRun) {
            if (c <= 8)
                launch_res_chunk<8>(h, d, c, n, stream, counters);
            else if (c <= 128)
                launch_res_chunk<128>(h, d, c, n, stream, counters);
            else
                launch_res_chunk<kMetroMaxJobs>(h, d, c, n, stream, counters);
        } else if (HEAT && GLR == 128) {
            if (c <= 8)
                launch_metro_chunk<8, 128, true>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, 128, true>(h, d, c, n, stream, counters, half);
        } else if (HEAT && GLR == kGeneralTile) {
            if (c <= 8)
                launch_metro_chunk<8, kGeneralTile, true>(h, d, c, n, stream, counters, half);
            else if (c <= 128)
                launch_metro_chunk<128, kGeneralTile, true>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, kGeneralTile, true>(h, d, c, n, stream,
                                                                      counters, half);
        } else if (HEAT && GLR == 64) {
            if (c <= 8)
                launch_metro_chunk<8, 64, true>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, 64, true>(h, d, c, n, stream, counters, half);
        } else if (HEAT) {
            if (c <= 1)
                launch_metro_chunk<1, 0, true>(h, d, c, n, stream, counters, half);
            else if (c <= 8)
                launch_metro_chunk<8, 0, true>(h, d, c, n, stream, counters, half);
            else if (c <= 128)
                launch_metro_chunk<128, 0, true>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, 0, true>(h, d, c, n, stream, counters, half);
        } else if (GLR == kGeneralTile) {
            if (c <= 8)
                launch_metro_chunk<8, kGeneralTile>(h, d, c, n, stream, counters, half);
            else if (c <= 128)
                launch_metro_chunk<128, kGeneralTile>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, kGeneralTile>(h, d, c, n, stream, counters, half);
        } else if (GLR == 128) {
            if (c <= 8)
                launch_metro_chunk<8, 128>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, 128>(h, d, c, n, stream, counters, half);
        } else if (GLR == 64) {
            if (c <= 8)
                launch_metro_chunk<8, 64>(h, d, c, n, stream, counters, half);
            else
                launch_metro_chunk<kMetroMaxJobs, 64>(h, d, c, n, stream, counters, half);
        } else if (c <= 1) {
            launch_metro_chunk<1, 0>(h, d, c, n, stream, counters, half);
        } else if (c <= 8) {
            launch_metro_chunk<8, 0>(h, d, c, n, stream, counters, half);
        } else if (c <= 32) {
            launch_metro_chunk<32, 0>(h, d, c, n, stream, counters, half);
        } else if (c <= 128) {
            launch_metro_chunk<128, 0>(h, d, c, n, stream, counters, half);
        } else {
            launch_metro_chunk<kMetroMaxJobs, 0>(h, d, c, n, stream, counters, half);
        }
    }
}

// A table read as runs, in this order: (with `resident`) the jobs marked for
// the sample-resident kernel, then those for the column kernels, then (with
// `general`) those of the general tile kernel, then side 64, then side 128
// (their own tile kernels).  A table in any other order is one run for the
// column kernel.
struct Run {
    int first, cnt, GLR;
};

static int split_runs(const JobDev *host, int n_jobs, bool general, bool resident, Run runs[5])
{
    constexpr int kCode[5] = {kResidentRun, 0, kGeneralTile, 64, 128};
    auto cls = [&](const JobDev &jd) {
        const int L = jd.geo.L;
        if (resident && jd.resident)
            return 0;
        return L == 64 ? 3 : L == 128 ? 4 : (general && general_tile_side(L)) ? 2 : 1;
    };
    int count[5] = {0, 0, 0, 0, 0};
    int prev = 0;
    for (int i = 0; i < n_jobs; ++i) {
        const int c = cls(host[i]);
        if (c < prev) {  // not in run order
            runs[0] = {0, n_jobs, 0};
            return 1;
        }
        prev = c;
        ++count[c];
    }
    int n_runs = 0, first = 0;
    for (int c = 0; c < 5; ++c)
        if (count[c] > 0) {
            runs[n_runs++] = {first, count[c], kCode[c]};
            first += count[c];
        }
    return n_runs;
}

cudaError_t launch_sweep_table(const JobDev *host0, const JobDev *dev0, int n_jobs0,
                               const JobDev *host1, const JobDev *dev1, int n_jobs1,
                               uint64_t n, cudaStream_t stream, unsigned long long *counters,
                               const SideStreams *side, int half, int streams)
{
    // Every run holds jobs of its own, so the runs need no order between them:
    // given side streams, run r goes to lane r mod (number of lanes), lane 0
    // being `stream` and the others side streams forked from it and joined
    // back after their n sweeps, so the runs share the GPU.  With fewer runs
    // than `streams`, runs are first split into runs of whole jobs: the blocks
    // of one run's launches then fill the SMs that another run's last wave
    // leaves idle.
    struct Item {
        Run run;
        bool heat;
    };
    Item items[10];
    int n_items = 0;
    Run runs[5];
    // the sample-resident kernel runs whole sweeps only
    int nr = split_runs(host0, n_jobs0, true, half < 0, runs);
    for (int r = 0; r < nr; ++r)
        items[n_items++] = {runs[r], false};
    nr = split_runs(host1, n_jobs1, true, false, runs);
    for (int r = 0; r < nr; ++r)
        items[n_items++] = {runs[r], true};
    const int lanes = side != nullptr ? 1 + kSideStreams : 1;
    const int want = std::min(std::max(streams, 1), lanes);
    // fewer runs than streams: halve the run of most jobs (whole jobs, the
    // first half keeps the larger share) until there are enough or none splits
    while (n_items < want) {
        int big = -1;
        for (int i = 0; i < n_items; ++i)
            if (items[i].run.cnt >= 2 && (big < 0 || items[i].run.cnt > items[big].run.cnt))
                big = i;
        if (big < 0)
            break;
        for (int i = n_items; i > big + 1; --i)
            items[i] = items[i - 1];
        const Run r = items[big].run;
        const int c0 = (r.cnt + 1) / 2;
        items[big].run = {r.first, c0, r.GLR};
        items[big + 1] = {{r.first + c0, r.cnt - c0, r.GLR}, items[big].heat};
        ++n_items;
    }
    const int used = std::min(n_items, lanes);
    const bool fork = used > 1;
    long shared = 0;
    if (fork)
        for (int i = 0; i < n_items; ++i) {
            const Run &r = items[i].run;
            if (r.GLR != 128 && r.GLR != 64 && r.GLR != kGeneralTile)
                continue;
            const JobDev *h = (items[i].heat ? host1 : host0) + r.first;
            for (int k = 0; k < r.cnt; ++k) {
                const int rows = (r.GLR == 64 || r.GLR == 128) ? h[k].row_hi - h[k].row_lo
                                                                : h[k].geo.n[1];
                shared += (long)h[k].n_samples * (h[k].geo.n[0] / 2) * (h[k].geo.n[2] / 2) * rows;
            }
        }
    if (fork) {
        cudaError_t err = cudaEventRecord(side->fork, stream);
        for (int r = 1; r < used && err == cudaSuccess; ++r)
            err = cudaStreamWaitEvent(side->stream[r - 1], side->fork, 0);
        if (err != cudaSuccess)
            return err;
    }
    t_tiles_shared = shared;
    for (int i = 0; i < n_items; ++i) {
        const int lane = i % used;
        cudaStream_t s = lane == 0 ? stream : side->stream[lane - 1];
        const Run &r = items[i].run;
        if (items[i].heat)
            launch_metro_run<true>(host1 + r.first, dev1 + r.first, r.cnt, r.GLR, n, s,
                                   counters, half);
        else
            launch_metro_run(host0 + r.first, dev0 + r.first, r.cnt, r.GLR, n, s, counters,
                             half);
    }
    t_tiles_shared = 0;
    if (fork) {
        cudaError_t err = cudaSuccess;
        for (int r = 1; r < used && err == cudaSuccess; ++r) {
            err = cudaEventRecord(side->join[r - 1], side->stream[r - 1]);
            if (err == cudaSuccess)
                err = cudaStreamWaitEvent(stream, side->join[r - 1], 0);
        }
        if (err != cudaSuccess)
            return err;
    }
    return cudaGetLastError();
}

void set_wait_policy(uint32_t limit, uint32_t mode)
{
    g_wait_limit = limit;
    g_wait_mode = mode;
}

cudaError_t read_sweep_status(cudaStream_t stream, uint32_t *status)
{
    unsigned int v = 0u, zero = 0u;
    cudaError_t err = cudaMemcpyFromSymbolAsync(&v, g_sweep_status, sizeof(v), 0,
                                                cudaMemcpyDeviceToHost, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyToSymbolAsync(g_sweep_status, &zero, sizeof(zero), 0,
                                      cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(stream);
    *status = v;
    return err;
}

cudaError_t prepare_resident_kernels()
{
    cudaError_t err = cudaSuccess;
    auto take = [&err](cudaError_t e) {
        if (err == cudaSuccess)
            err = e;
    };
    take(res_opt_in<false, 8>());
    take(res_opt_in<true, 8>());
    take(res_opt_in<false, 128>());
    take(res_opt_in<true, 128>());
    take(res_opt_in<false, kMetroMaxJobs>());
    take(res_opt_in<true, kMetroMaxJobs>());
    return err;
}

cudaError_t launch_advance_time(JobDev *jobs_dev, int n_jobs, uint64_t n, cudaStream_t stream)
{
    if (n_jobs <= 0)
        return cudaSuccess;
    advance_time_kernel<<<(n_jobs + 127) / 128, 128, 0, stream>>>(jobs_dev, n_jobs, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ea
