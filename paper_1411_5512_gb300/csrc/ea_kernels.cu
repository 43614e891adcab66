// ea_kernels.cu -- sm_103a kernels of the EA ageing library.
//
// All state is bit-packed: one 32-bit word holds up to 32 sites of ONE sample
// (Geo in ea_internal.h), so every lane of a word shares one temperature and
// one Philox key, and a per-sample reduction is a plain popcount of words.
//
// The update of a word is pure bitwise logic (Sec. III: "bit operations are
// used to perform the update for all bit-coded spins at the same time"):
//   unsatisfied-bond bits  u_j = s ^ n_j ^ J_j                      (6 LOP3)
//   bit-sliced count of the six u_j -> (b2 b1 b0) = u in 0..6       (8 LOP3)
//   dE = 12 - 4u (Eq. 9); Metropolis accepts u >= 3 outright and compares a
//   64-bit uniform r against the integer threshold of dE otherwise.
// The comparison r < thr is done bit-sliced from the most significant bit:
// plane k of the Philox stream gives bit 63-k of r for all 32 lanes at once;
// a lane is decided at the first plane where its r bit differs from its
// threshold bit, so most words finish after one or two Philox calls.
#include <cstdint>

#include "ea_internal.h"

namespace ea {
namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplies (0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85) between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

constexpr uint32_t kStreamCouplings = 0u << 30;
constexpr uint32_t kStreamSpins = 1u << 30;
constexpr uint32_t kStreamSweep = 2u << 30;

// c ? x : y, bitwise
__device__ __forceinline__ uint32_t sel(uint32_t c, uint32_t x, uint32_t y)
{
    return (c & x) | (~c & y);
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c)
{
    return (a & b) | (a & c) | (b & c);
}

// Neighbour word read across the periodic wrap of axis d (dir 0: +1, 1: -1).
__device__ __forceinline__ uint32_t realign(uint32_t w, const Geo &g, int d, int dir)
{
    return ((w >> g.sA[d][dir]) & g.mA[d][dir]) | ((w << g.sB[d][dir]) & g.mB[d][dir]);
}

__device__ __forceinline__ void word_coords(const Geo &g, int w, int &xw, int &yw, int &zw)
{
    xw = w % g.n[0];
    const int r = w / g.n[0];
    yw = r % g.n[1];
    zw = r / g.n[1];
}

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------
__global__ void init_couplings_kernel(uint32_t *__restrict__ J, Geo g, uint64_t thr_p, uint32_t k0,
                                      uint32_t k1)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    uint32_t jw[3] = {0u, 0u, 0u};
    for (int b = 0; b < g.lanes; ++b) {
        const int bx = b % g.k[0], by = (b / g.k[0]) % g.k[1], bz = b / (g.k[0] * g.k[1]);
        const uint32_t x = bx * g.n[0] + xw, y = by * g.n[1] + yw, z = bz * g.n[2] + zw;
        const uint32_t i = x + (uint32_t)g.L * (y + (uint32_t)g.L * z);
        const uint4 o = philox10(make_uint4(i, 0u, kStreamCouplings, (uint32_t)s), k0, k1);
        jw[0] |= (uint32_t)((uint64_t)o.x < thr_p) << b;
        jw[1] |= (uint32_t)((uint64_t)o.y < thr_p) << b;
        jw[2] |= (uint32_t)((uint64_t)o.z < thr_p) << b;
    }
    const size_t W = (size_t)g.words;
    uint32_t *Js = J + (size_t)s * 3 * W;
    Js[w] = jw[0];
    Js[W + w] = jw[1];
    Js[2 * W + w] = jw[2];
}

__global__ void init_spins_kernel(uint32_t *__restrict__ spins, Geo g, uint32_t k0, uint32_t k1)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    uint32_t rep[2] = {0u, 0u};
    for (int b = 0; b < g.lanes; ++b) {
        const int bx = b % g.k[0], by = (b / g.k[0]) % g.k[1], bz = b / (g.k[0] * g.k[1]);
        const uint32_t x = bx * g.n[0] + xw, y = by * g.n[1] + yw, z = bz * g.n[2] + zw;
        const uint32_t i = x + (uint32_t)g.L * (y + (uint32_t)g.L * z);
        const uint4 o = philox10(make_uint4(i, 0u, kStreamSpins, (uint32_t)s), k0, k1);
        rep[0] |= (o.x >> 31) << b;
        rep[1] |= (o.y >> 31) << b;
    }
    const int c = (xw + yw + zw) & 1;
    const size_t W = (size_t)g.words;
    uint32_t *Ss = spins + (size_t)s * 2 * W;
    Ss[w] = rep[0 ^ c];      // area 0 holds replica (0 XOR colour)
    Ss[W + w] = rep[1 ^ c];  // area 1 holds replica (1 XOR colour)
}

// ---------------------------------------------------------------------------
// half-step update
// ---------------------------------------------------------------------------
template <int RULE>
struct RuleInfo;
template <>
struct RuleInfo<0> {
    static constexpr int NT = 3;  // thresholds of u = 0, 1, 2 (dE = 12, 8, 4)
};
template <>
struct RuleInfo<1> {
    static constexpr int NT = 7;  // thresholds of u = 0..6
};

// bitwise 8-way select on (b2 b1 b0) of the values f[0..6] (f[7] = 0)
__device__ __forceinline__ uint32_t mux7(uint32_t b2, uint32_t b1, uint32_t b0, uint32_t f0,
                                         uint32_t f1, uint32_t f2, uint32_t f3, uint32_t f4,
                                         uint32_t f5, uint32_t f6)
{
    const uint32_t m0 = sel(b0, f1, f0), m1 = sel(b0, f3, f2), m2 = sel(b0, f5, f4),
                   m3 = ~b0 & f6;
    return sel(b2, sel(b1, m3, m2), sel(b1, m1, m0));
}

template <int RULE>
__global__ void __launch_bounds__(256) halfstep_kernel(SweepLaunch p, int h, uint64_t t)
{
    constexpr int NT = RuleInfo<RULE>::NT;
    // s_tm[call][u] = the four plane masks (all-ones where the threshold bit is 1)
    __shared__ uint4 s_tm[16][NT];
    for (int idx = threadIdx.x; idx < 16 * NT * 4; idx += blockDim.x) {
        const int call = idx / (NT * 4), u = (idx / 4) % NT, j = idx % 4;
        const int k = 4 * call + j;
        const uint32_t bit = (uint32_t)(p.thr.thr_u[u] >> (63 - k)) & 1u;
        reinterpret_cast<uint32_t *>(s_tm)[idx] = 0u - bit;
    }
    __syncthreads();

    const Geo &g = p.geo;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    const int c = (xw + yw + zw) & 1;
    const int a = h ^ c;  // replica updated at this word-site in half-step h

    const size_t W = (size_t)g.words;
    uint32_t *upd = p.spins + ((size_t)s * 2 + h) * W;
    const uint32_t *__restrict__ nb = p.spins + ((size_t)s * 2 + (h ^ 1)) * W;
    const uint32_t *__restrict__ Jx = p.J + (size_t)s * 3 * W;
    const uint32_t *__restrict__ Jy = Jx + W;
    const uint32_t *__restrict__ Jz = Jy + W;

    const uint32_t sp = upd[w];
    const int sy = g.n[0], sz = g.n[0] * g.n[1];
    uint32_t nxp, nxm, jxm, nyp, nym, jym, nzp, nzm, jzm;
    if (xw + 1 < g.n[0])
        nxp = nb[w + 1];
    else
        nxp = realign(nb[w - (g.n[0] - 1)], g, 0, 0);
    if (xw > 0) {
        nxm = nb[w - 1];
        jxm = Jx[w - 1];
    } else {
        nxm = realign(nb[w + (g.n[0] - 1)], g, 0, 1);
        jxm = realign(Jx[w + (g.n[0] - 1)], g, 0, 1);
    }
    if (yw + 1 < g.n[1])
        nyp = nb[w + sy];
    else
        nyp = realign(nb[w - (g.n[1] - 1) * sy], g, 1, 0);
    if (yw > 0) {
        nym = nb[w - sy];
        jym = Jy[w - sy];
    } else {
        nym = realign(nb[w + (g.n[1] - 1) * sy], g, 1, 1);
        jym = realign(Jy[w + (g.n[1] - 1) * sy], g, 1, 1);
    }
    if (zw + 1 < g.n[2])
        nzp = nb[w + sz];
    else
        nzp = realign(nb[w - (g.n[2] - 1) * sz], g, 2, 0);
    if (zw > 0) {
        nzm = nb[w - sz];
        jzm = Jz[w - sz];
    } else {
        nzm = realign(nb[w + (g.n[2] - 1) * sz], g, 2, 1);
        jzm = realign(Jz[w + (g.n[2] - 1) * sz], g, 2, 1);
    }

    // unsatisfied bonds and their bit-sliced count u = 4 b2 + 2 b1 + b0
    const uint32_t u0 = sp ^ nxp ^ Jx[w], u1 = sp ^ nxm ^ jxm;
    const uint32_t u2 = sp ^ nyp ^ Jy[w], u3 = sp ^ nym ^ jym;
    const uint32_t u4 = sp ^ nzp ^ Jz[w], u5 = sp ^ nzm ^ jzm;
    const uint32_t s1 = u0 ^ u1 ^ u2, c1 = maj3(u0, u1, u2);
    const uint32_t s2 = u3 ^ u4 ^ u5, c2 = maj3(u3, u4, u5);
    const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t b1 = c1 ^ c2 ^ c3, b2 = maj3(c1, c2, c3);

    uint32_t alw;
    if (RULE == 0) {
        alw = b2 | (b1 & b0);  // u >= 3 <=> dE <= 0
    } else {
        const uint32_t f = p.thr.always_u;
        alw = mux7(b2, b1, b0, 0u - (f & 1u), 0u - ((f >> 1) & 1u), 0u - ((f >> 2) & 1u),
                   0u - ((f >> 3) & 1u), 0u - ((f >> 4) & 1u), 0u - ((f >> 5) & 1u),
                   0u - ((f >> 6) & 1u));
    }
    uint32_t flip;
    if (p.thr.all_always) {
        flip = ~0u;
    } else if (p.thr.none_random) {
        flip = alw;
    } else {
        uint32_t U = ~alw & g.valid;  // lanes still comparing r with their threshold
        uint32_t A = 0u;              // lanes accepted by the comparison
        const uint32_t c2base =
            kStreamSweep | (((uint32_t)(t >> 32) & 0xFFFFu) << 8) | ((uint32_t)a << 4);
        const uint32_t c3 = (uint32_t)(s / p.rng_group);
        for (int call = 0; call < 16 && U != 0u; ++call) {
            const uint4 R =
                philox10(make_uint4((uint32_t)w, (uint32_t)t, c2base | (uint32_t)call, c3), p.key0,
                         p.key1);
            if ((p.thr.zero_calls >> call) & 1u) {
                // every needed threshold bit is 0 on these planes: a 1 bit rejects
                U &= ~(R.x | R.y | R.z | R.w);
                continue;
            }
            uint32_t tk[4];
            if (RULE == 0) {
                const uint4 T0 = s_tm[call][0], T1 = s_tm[call][1], T2 = s_tm[call][2];
                tk[0] = sel(b1, T2.x, sel(b0, T1.x, T0.x));
                tk[1] = sel(b1, T2.y, sel(b0, T1.y, T0.y));
                tk[2] = sel(b1, T2.z, sel(b0, T1.z, T0.z));
                tk[3] = sel(b1, T2.w, sel(b0, T1.w, T0.w));
            } else {
                uint4 T[7];
#pragma unroll
                for (int u = 0; u < 7; ++u)
                    T[u] = s_tm[call][u];
                tk[0] = mux7(b2, b1, b0, T[0].x, T[1].x, T[2].x, T[3].x, T[4].x, T[5].x, T[6].x);
                tk[1] = mux7(b2, b1, b0, T[0].y, T[1].y, T[2].y, T[3].y, T[4].y, T[5].y, T[6].y);
                tk[2] = mux7(b2, b1, b0, T[0].z, T[1].z, T[2].z, T[3].z, T[4].z, T[5].z, T[6].z);
                tk[3] = mux7(b2, b1, b0, T[0].w, T[1].w, T[2].w, T[3].w, T[4].w, T[5].w, T[6].w);
            }
            const uint32_t r[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                A |= U & ~r[j] & tk[j];   // r bit 0 < threshold bit 1: accept
                U &= ~(r[j] ^ tk[j]);     // bits differ: decided
            }
        }
        flip = alw | A;
    }
    upd[w] = sp ^ (flip & g.valid);
}

// ---------------------------------------------------------------------------
// observables: popcount sums, block-reduced, accumulated with integer atomics
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v)
{
    __shared__ unsigned long long s_part[32];
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        s_part[wid] = v;
    __syncthreads();
    unsigned long long tot = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i)
            tot += s_part[i];
    }
    return tot;
}

// q_pop[s] += popc(area0 ^ area1) (= number of sites where the replicas differ);
// u_pop[s][a] += unsatisfied bonds of replica a.
__global__ void obs_state_kernel(const uint32_t *__restrict__ spins, const uint32_t *__restrict__ J,
                                 Geo g, unsigned long long *q_pop, unsigned long long *u_pop)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const size_t W = (size_t)g.words;
    unsigned long long q = 0, ua[2] = {0, 0};
    if (w < g.words) {
        int xw, yw, zw;
        word_coords(g, w, xw, yw, zw);
        const int c = (xw + yw + zw) & 1;
        const uint32_t *area[2] = {spins + (size_t)s * 2 * W, spins + ((size_t)s * 2 + 1) * W};
        const uint32_t *Js = J + (size_t)s * 3 * W;
        q = __popc(area[0][w] ^ area[1][w]);
        const int step[3] = {1, g.n[0], g.n[0] * g.n[1]};
        const int coord[3] = {xw, yw, zw};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const uint32_t sa = area[a ^ c][w];
            const uint32_t *nbarea = area[a ^ c ^ 1];  // replica a at the other colour
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                uint32_t nbw;
                if (coord[d] + 1 < g.n[d])
                    nbw = nbarea[w + step[d]];
                else
                    nbw = realign(nbarea[w - (g.n[d] - 1) * step[d]], g, d, 0);
                ua[a] += __popc((sa ^ nbw ^ Js[d * W + w]) & g.valid);
            }
        }
    }
    const unsigned long long tq = block_sum(q);
    if (threadIdx.x == 0 && tq)
        atomicAdd(&q_pop[s], tq);
    const unsigned long long t0 = block_sum(ua[0]);
    if (threadIdx.x == 0 && t0)
        atomicAdd(&u_pop[2 * s], t0);
    const unsigned long long t1 = block_sum(ua[1]);
    if (threadIdx.x == 0 && t1)
        atomicAdd(&u_pop[2 * s + 1], t1);
}

// a_pop[s][a] += sites where replica a differs from its snapshot
__global__ void obs_autocorr_kernel(const uint32_t *__restrict__ snap,
                                    const uint32_t *__restrict__ spins, Geo g,
                                    unsigned long long *a_pop)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const size_t W = (size_t)g.words;
    unsigned long long d[2] = {0, 0};
    if (w < g.words) {
        int xw, yw, zw;
        word_coords(g, w, xw, yw, zw);
        const int c = (xw + yw + zw) & 1;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const size_t off = ((size_t)s * 2 + (a ^ c)) * W + w;
            d[a] = __popc(snap[off] ^ spins[off]);
        }
    }
    const unsigned long long t0 = block_sum(d[0]);
    if (threadIdx.x == 0 && t0)
        atomicAdd(&a_pop[2 * s], t0);
    const unsigned long long t1 = block_sum(d[1]);
    if (threadIdx.x == 0 && t1)
        atomicAdd(&a_pop[2 * s + 1], t1);
}

__device__ __forceinline__ uint32_t low_bits(int n)
{
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// g_pop[s][d][r] += sites i where q_i != q_{i + r e_d}, q = replica 0 XOR 1
__global__ void obs_c4_kernel(const uint32_t *__restrict__ spins, Geo g,
                              unsigned long long *g_pop)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const int R = g.L / 2 + 1;
    const int d = blockIdx.z / R, r = blockIdx.z % R;
    const size_t W = (size_t)g.words;
    unsigned long long cnt = 0;
    if (w < g.words) {
        const uint32_t *A0 = spins + (size_t)s * 2 * W, *A1 = A0 + W;
        int xw, yw, zw;
        word_coords(g, w, xw, yw, zw);
        const int coord[3] = {xw, yw, zw};
        const int step[3] = {1, g.n[0], g.n[0] * g.n[1]};
        const int nd = g.n[d], kd = g.k[d], st = g.stride[d];
        const int m = coord[d] + r;
        const int w2 = w + (m % nd - coord[d]) * step[d];
        const int qrot = (m / nd) % kd;  // block-index shift of every lane
        const uint32_t q = A0[w] ^ A1[w];
        uint32_t q2 = A0[w2] ^ A1[w2];
        if (qrot != 0) {
            // lane with block index b_d reads lane b_d + qrot (mod kd)
            const int period = st * kd;
            const uint32_t base = low_bits((kd - qrot) * st);
            uint32_t mA = 0;
            for (int j = 0; j < g.lanes; j += period)
                mA |= base << j;
            mA &= g.valid;
            const uint32_t mB = g.valid & ~mA;
            q2 = ((q2 >> (qrot * st)) & mA) | ((q2 << ((kd - qrot) * st)) & mB);
        }
        cnt = __popc(q ^ q2);
    }
    const unsigned long long tot = block_sum(cnt);
    if (threadIdx.x == 0 && tot)
        atomicAdd(&g_pop[((size_t)s * 3 + d) * R + r], tot);
}

constexpr int kBlock = 256;

inline dim3 grid_for(const Geo &g, int n_samples, int z = 1)
{
    return dim3((unsigned)((g.words + kBlock - 1) / kBlock), (unsigned)n_samples, (unsigned)z);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_init_couplings(uint32_t *J, const Geo &g, int n_samples, double p_neg,
                                  uint64_t seed, cudaStream_t stream)
{
    const uint64_t thr_p =
        p_neg >= 1.0 ? ((uint64_t)1 << 32) : (uint64_t)floor(ldexp(p_neg, 32));
    init_couplings_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(
        J, g, thr_p, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_init_spins(uint32_t *spins, const Geo &g, int n_samples, uint64_t seed,
                              cudaStream_t stream)
{
    init_spins_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(spins, g, (uint32_t)seed,
                                                                     (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_sweeps(const SweepLaunch &p, uint64_t t0, uint64_t n, cudaStream_t stream)
{
    const dim3 grid = grid_for(p.geo, p.n_samples);
    for (uint64_t k = 0; k < n; ++k) {
        for (int h = 0; h < 2; ++h) {
            if (p.thr.rule == 0)
                halfstep_kernel<0><<<grid, kBlock, 0, stream>>>(p, h, t0 + k);
            else
                halfstep_kernel<1><<<grid, kBlock, 0, stream>>>(p, h, t0 + k);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_obs_state(const uint32_t *spins, const uint32_t *J, const Geo &g, int n_samples,
                             unsigned long long *q_pop, unsigned long long *u_pop,
                             cudaStream_t stream)
{
    obs_state_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(spins, J, g, q_pop, u_pop);
    return cudaGetLastError();
}

cudaError_t launch_obs_autocorr(const uint32_t *snap, const uint32_t *spins, const Geo &g,
                                int n_samples, unsigned long long *a_pop, cudaStream_t stream)
{
    obs_autocorr_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(snap, spins, g, a_pop);
    return cudaGetLastError();
}

cudaError_t launch_obs_c4(const uint32_t *spins, const Geo &g, int n_samples,
                          unsigned long long *g_pop, cudaStream_t stream)
{
    const int R = g.L / 2 + 1;
    obs_c4_kernel<<<grid_for(g, n_samples, 3 * R), kBlock, 0, stream>>>(spins, g, g_pop);
    return cudaGetLastError();
}

}  // namespace ea
