// ea_kernels.cu -- initial-state and observable kernels of the EA ageing library
// (the sweep kernel is in ea_sweep.cu).
//
// All state is bit-packed: one 32-bit word holds up to 32 sites of ONE sample
// (Geo in ea_internal.h), so a per-sample reduction is a plain popcount of
// words: sum_i S_i S'_i = N - 2 * (number of differing bits).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ea_device.cuh"
#include "ea_internal.h"

namespace ea {
namespace {

using dev::kStreamCouplings;
using dev::kStreamSpins;
using dev::philox10;

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

// The site index i = x + L (y + L z) of each lane b of word-site (xw, yw, zw),
// lane b = bx + k0 (by + k1 bz) at (bx n0 + xw, by n1 + yw, bz n2 + zw), in
// lane order without divisions.
struct LaneSites {
    const Geo &g;
    int bx = 0, by = 0;
    uint32_t i;
    __device__ LaneSites(const Geo &geo, int xw, int yw, int zw)
        : g(geo), i((uint32_t)xw + (uint32_t)geo.L * ((uint32_t)yw + (uint32_t)geo.L * (uint32_t)zw))
    {
    }
    __device__ void next()
    {
        const uint32_t L = (uint32_t)g.L;
        i += (uint32_t)g.n[0];
        if (++bx < g.k[0])
            return;
        bx = 0;
        i += L * (uint32_t)g.n[1] - L;  // x back to xw, y one block on
        if (++by < g.k[1])
            return;
        by = 0;
        i += L * L * (uint32_t)g.n[2] - L * L;  // y back to yw, z one block on
    }
};

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------
__global__ void init_couplings_kernel(uint32_t *__restrict__ J, Geo g, uint64_t thr_p, uint32_t k0,
                                      uint32_t k1, uint32_t s0)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;  // the context's sample s is the job's sample s0 + s
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    uint32_t jw[3] = {0u, 0u, 0u};
    LaneSites ls(g, xw, yw, zw);
    for (int b = 0; b < g.lanes; ++b, ls.next()) {
        const uint32_t i = ls.i;
        const uint4 o = philox10(make_uint4(i, 0u, kStreamCouplings, s0 + (uint32_t)s), k0, k1);
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

// ---------------------------------------------------------------------------
// Couplings with an exact count: the negative bonds are the first K in the
// order of (key, b), b = d N + i, key = (out0 << 32) | out1 of
// Philox(ctr = (i, 1 + d, 0, s)).  The K-th element of that order is found
// by a radix select over the 96-bit composite (key, b), 8 bits per pass, most
// significant first: a pass counts the bonds whose higher digits match the
// prefix found so far, and a one-block step picks the digit where the count
// reaches the remaining rank.  Per sample, state = {prefix[3], rank left}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bond_key(uint32_t i, int d, uint32_t s, uint32_t k0, uint32_t k1,
                                        uint32_t &hi, uint32_t &lo)
{
    const uint4 o = philox10(make_uint4(i, 1u + (uint32_t)d, kStreamCouplings, s), k0, k1);
    hi = o.x;
    lo = o.y;
}

__global__ void exact_hist_kernel(int L, int pass, const uint32_t *__restrict__ state,
                                  uint32_t *__restrict__ hist, uint32_t k0, uint32_t k1,
                                  uint32_t s0)
{
    __shared__ uint32_t h[256];
    const uint32_t s = blockIdx.y;
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        h[i] = 0u;
    __syncthreads();
    const uint64_t N = (uint64_t)L * L * L;
    const int wsel = pass >> 2, shift = 24 - 8 * (pass & 3);
    const uint32_t *st = state + (size_t)s * 4;
    const uint32_t P[3] = {st[0], st[1], st[2]};
    // bits of word wsel above the digit must match; words before it too
    const uint32_t above = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < 3 * N;
         b += (uint64_t)gridDim.x * blockDim.x) {
        const int d = (int)(b / N);
        const uint32_t i = (uint32_t)(b - (uint64_t)d * N);
        uint32_t c[3];
        bond_key(i, d, s0 + s, k0, k1, c[0], c[1]);
        c[2] = (uint32_t)b;
        bool match = true;
        for (int w = 0; w < wsel; ++w)
            match = match && c[w] == P[w];
        match = match && ((c[wsel] ^ P[wsel]) & above) == 0u;
        if (match)
            atomicAdd(&h[(c[wsel] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i])
            atomicAdd(&hist[(size_t)s * 256 + i], h[i]);
}

// One block of 256 threads per sample: the digit where the running count
// reaches the rank left; clears the histogram for the next pass.
__global__ void exact_select_kernel(int pass, uint32_t *__restrict__ state,
                                    uint32_t *__restrict__ hist)
{
    __shared__ uint32_t cum[256];
    const uint32_t s = blockIdx.x;
    uint32_t *st = state + (size_t)s * 4;
    uint32_t *hs = hist + (size_t)s * 256;
    const int t = threadIdx.x;
    const uint32_t cnt = hs[t];
    cum[t] = cnt;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {  // inclusive scan
        const uint32_t v = t >= off ? cum[t - off] : 0u;
        __syncthreads();
        cum[t] += v;
        __syncthreads();
    }
    const uint32_t krem = st[3];
    const uint32_t before = cum[t] - cnt;
    if (cnt > 0u && before < krem && krem <= cum[t]) {
        const int wsel = pass >> 2, shift = 24 - 8 * (pass & 3);
        st[wsel] |= (uint32_t)t << shift;
        st[3] = krem - before;
    }
    hs[t] = 0u;
}

// J words from the K-th composite P: a bond is negative iff (key, b) <= P.
__global__ void exact_mark_kernel(uint32_t *__restrict__ J, Geo g, const uint32_t *__restrict__ state,
                                  int none, uint32_t k0, uint32_t k1, uint32_t s0)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    const uint32_t *st = state + (size_t)s * 4;
    const uint32_t P0 = st[0], P1 = st[1], P2 = st[2];
    const uint64_t N = (uint64_t)g.L * g.L * g.L;
    uint32_t jw[3] = {0u, 0u, 0u};
    if (!none) {
        LaneSites ls(g, xw, yw, zw);
        for (int b = 0; b < g.lanes; ++b, ls.next()) {
            const uint32_t i = ls.i;
            for (int d = 0; d < 3; ++d) {
                uint32_t hi, lo;
                bond_key(i, d, s0 + (uint32_t)s, k0, k1, hi, lo);
                const uint32_t bi = (uint32_t)((uint64_t)d * N + i);
                const bool le = hi != P0 ? hi < P0 : (lo != P1 ? lo < P1 : bi <= P2);
                jw[d] |= (uint32_t)le << b;
            }
        }
    }
    const size_t W = (size_t)g.words;
    uint32_t *Js = J + (size_t)s * 3 * W;
    Js[w] = jw[0];
    Js[W + w] = jw[1];
    Js[2 * W + w] = jw[2];
}

__global__ void init_spins_kernel(uint32_t *__restrict__ spins, Geo g, uint32_t k0, uint32_t k1,
                                  uint32_t s0)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (w >= g.words)
        return;
    int xw, yw, zw;
    word_coords(g, w, xw, yw, zw);
    uint32_t rep[2] = {0u, 0u};
    LaneSites ls(g, xw, yw, zw);
    for (int b = 0; b < g.lanes; ++b, ls.next()) {
        const uint32_t i = ls.i;
        const uint4 o = philox10(make_uint4(i, 0u, kStreamSpins, s0 + (uint32_t)s), k0, k1);
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
// observables: popcount sums, block-reduced, accumulated with integer atomics
// ---------------------------------------------------------------------------
// Everything a measurement time takes from the current state, in one pass over
// it: q_pop[s] += popc(area0 ^ area1) (the sites where the replicas differ),
// u_pop[s][a] += the unsatisfied bonds of replica a, and for each listed
// snapshot a_pop[k][s][a] += the sites where replica a differs from it.  With
// q_pop NULL only the snapshot comparisons run (a list longer than one
// launch holds).
__global__ void __launch_bounds__(kObsThreads)
    obs_time_kernel(const __grid_constant__ ObsTimeParams P, Geo g)
{
    constexpr int kAcc = 3 + 2 * kObsMaxSnaps;
    const int s = blockIdx.y;
    const size_t W = (size_t)g.words;
    const uint32_t *__restrict__ area0 = P.spins + (size_t)s * 2 * W;
    const uint32_t *__restrict__ area1 = area0 + W;
    const uint32_t *__restrict__ Js = P.J + (size_t)s * 3 * W;
    const bool state = P.q_pop != nullptr;
    uint32_t acc[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i)
        acc[i] = 0u;
    const int step[3] = {1, g.n[0], g.n[0] * g.n[1]};
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < g.words;
         w += gridDim.x * blockDim.x) {
        int xw, yw, zw;
        word_coords(g, w, xw, yw, zw);
        const int c = (xw + yw + zw) & 1;  // area h at w holds replica h ^ c
        const uint32_t cur[2] = {area0[w], area1[w]};
        if (state) {
            acc[0] += __popc(cur[0] ^ cur[1]);
            const int coord[3] = {xw, yw, zw};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const uint32_t sa = cur[a ^ c];
                const uint32_t *nbarea = (a ^ c) ? area0 : area1;  // replica a, other colour
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const uint32_t nbw = coord[d] + 1 < g.n[d]
                                             ? nbarea[w + step[d]]
                                             : realign(nbarea[w - (g.n[d] - 1) * step[d]], g, d, 0);
                    acc[1 + a] += __popc((sa ^ nbw ^ Js[d * W + w]) & g.valid);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kObsMaxSnaps; ++k) {
            if (k < P.n_snap) {
                const uint32_t *__restrict__ sn = P.snap[k] + (size_t)s * 2 * W;
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    acc[3 + 2 * k + a] += __popc(sn[(size_t)(a ^ c) * W + w] ^ cur[a ^ c]);
            }
        }
    }
    // one block reduction for all accumulators: warps first, then one thread each
    __shared__ unsigned long long s_part[kAcc][kObsThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_acc = 3 + 2 * P.n_snap;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) {
        if (i < n_acc) {
            unsigned long long v = acc[i];
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0)
                s_part[i][wid] = v;
        }
    }
    __syncthreads();
    const int i = (int)threadIdx.x;
    if (i < n_acc && (i >= 3 || state)) {
        unsigned long long tot = 0;
        for (int k = 0; k < kObsThreads / 32; ++k)
            tot += s_part[i][k];
        unsigned long long *dst = i == 0  ? P.q_pop + s
                                  : i < 3 ? P.u_pop + 2 * s + (i - 1)
                                          : P.a_pop[(i - 3) / 2] + 2 * s + ((i - 3) & 1);
        if (tot)
            atomicAdd(dst, tot);
    }
}

__device__ __forceinline__ uint32_t low_bits(int n)
{
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// g_pop[s][d][r] += sites i where q_i != q_{i + r e_d}, q = replica 0 XOR 1
// (the overlap field of Eq. 2; its correlation along the axes is Eq. 3).
//
// A block stages whole word-lines along axis d (n_d words each, every word a
// bundle of 32 / k_d lattice lines) as q in shared memory; thread r then sums,
// over the staged lines, popc(q[i] ^ q[i + r]) with the lanes realigned where
// the shift crosses the periodic wrap of the word lattice: for r = A n_d + B,
// positions i + B < n_d read word i + B rotated by A blocks, the others word
// i + B - n_d rotated by A + 1 blocks (mod k_d).
constexpr int kC4Words = 2048;  // staged words per block


// out[b] = in[b with block index b_d + q (mod k)] for the lanes of axis d
struct Rot {
    int sA, sB;
    uint32_t mA, mB;
};

__device__ __forceinline__ Rot make_rot(const Geo &g, int d, int q)
{
    Rot r;
    const int k = g.k[d], st = g.stride[d];
    q %= k;
    if (q == 0) {
        r.sA = 0;
        r.sB = 0;
        r.mA = g.valid;
        r.mB = 0u;
        return r;
    }
    const int period = st * k;
    const uint32_t base = low_bits((k - q) * st);
    uint32_t mA = 0u;
    for (int j = 0; j < g.lanes; j += period)
        mA |= base << j;
    r.mA = mA & g.valid;
    r.mB = g.valid & ~r.mA;
    r.sA = q * st;
    r.sB = (k - q) * st;
    return r;
}

__device__ __forceinline__ uint32_t rot(uint32_t w, const Rot &r)
{
    return ((w >> r.sA) & r.mA) | ((w << r.sB) & r.mB);
}

__global__ void __launch_bounds__(256) obs_c4_kernel(const uint32_t *__restrict__ spins, Geo g,
                                                     unsigned long long *g_pop)
{
    __shared__ uint32_t s_q[kC4Words];
    const int d = blockIdx.y;
    const int s = blockIdx.z;
    const int nd = g.n[d];
    const int n_lines = g.words / nd;
    const int lines_per_block = kC4Words / nd > 0 ? kC4Words / nd : 1;
    const int l0 = blockIdx.x * lines_per_block;
    const int nl = min(lines_per_block, n_lines - l0);  // <= 0: nothing for this block
    const size_t W = (size_t)g.words;
    const uint32_t *A0 = spins + (size_t)s * 2 * W, *A1 = A0 + W;
    // word index of position i of line l along axis d
    const int n0 = g.n[0], n1 = g.n[1];
    auto word_of = [&](int l, int i) -> int {
        if (d == 0)
            return i + n0 * l;                      // l = y' + n1 z'
        if (d == 1)
            return (l % n0) + n0 * (i + n1 * (l / n0));  // l = x' + n0 z'
        return l + n0 * n1 * i;                     // l = x' + n0 y'
    };
    for (int e = threadIdx.x; e < nl * nd; e += blockDim.x) {
        const int l = e / nd, i = e - l * nd;
        const int w = word_of(l0 + l, i);
        s_q[e] = A0[w] ^ A1[w];
    }
    __syncthreads();
    const int R = g.L / 2 + 1;
    // thread (group gi, shift r): the lane rotations of r are set up once, and
    // the groups split the staged lines between them
    const int groups = blockDim.x / R > 0 ? blockDim.x / R : 1;
    for (int task = threadIdx.x; task < groups * R; task += blockDim.x) {
        const int gi = task / R, r = task - gi * R;
        const int A = r / nd, B = r - A * nd;
        const Rot r0 = make_rot(g, d, A), r1 = make_rot(g, d, A + 1);
        unsigned long long cnt = 0;
        for (int l = gi; l < nl; l += groups) {
            const uint32_t *q = s_q + l * nd;
            unsigned int c = 0;
            for (int i = 0; i < nd - B; ++i)
                c += __popc(q[i] ^ rot(q[i + B], r0));
            for (int i = nd - B; i < nd; ++i)
                c += __popc(q[i] ^ rot(q[i + B - nd], r1));
            cnt += c;
        }
        if (cnt)
            atomicAdd(&g_pop[((size_t)s * 3 + d) * R + r], cnt);
    }
}

// The four-point sums of a side whose word lattice holds all 32 lanes along z
// (kx = ky = 1, kz = 32; here L = 64 or 128).  x and y shifts move whole words,
// a z shift by r = A n2 + B rotates the lanes by A (A + 1 across the wrap).
// Grid (tiles, 3 axes, samples), 8 warps per block:
//   x: a warp per line (y', z'), staged twice in shared memory so that a
//      shift needs no wrap;
//   y: a block per tile of 32 x-columns at one z', staged with a padded row
//      (no bank conflicts along y) and doubled along y; a warp per 4 columns;
//   z: a thread per column (x', y'), its N2 words in registers.
// Each lane sums the popcounts of its words for one shift, the warp adds them
// up with one reduction, and the block adds its totals into g_pop.
constexpr int kC4FastMaxL = 128;

template <int N2>
__global__ void __launch_bounds__(256) obs_c4_fast_kernel(const uint32_t *__restrict__ spins,
                                                          Geo g, unsigned long long *g_pop)
{
    const int d = blockIdx.y, s = blockIdx.z;
    const int L = g.L, R = L / 2 + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t W = (size_t)g.words;
    const uint32_t *__restrict__ A0 = spins + (size_t)s * 2 * W;
    const uint32_t *__restrict__ A1 = A0 + W;
    __shared__ uint32_t s_buf[2 * kC4FastMaxL * 33];   // lines (x) or a padded tile (y)
    __shared__ unsigned int s_acc[8][kC4FastMaxL / 2 + 1];
    for (int i = threadIdx.x; i < 8 * R; i += blockDim.x)
        s_acc[i / R][i % R] = 0u;
    __syncthreads();
    const int n0 = L, n1 = L;  // words along x and y
    if (d == 0) {
        // lines (y', z') of n0 words, one per warp
        const int n_lines = n1 * N2;
        const int l = blockIdx.x * 8 + warp;
        if (blockIdx.x * 8 < n_lines && l < n_lines) {
            uint32_t *line = s_buf + warp * 2 * n0;
            const int base = l * n0;  // word of x' = 0 on this line
            uint32_t q[kC4FastMaxL / 32];
#pragma unroll
            for (int k = 0; k < kC4FastMaxL / 32; ++k) {
                if (k * 32 < n0) {
                    const int x = lane + 32 * k;
                    q[k] = A0[base + x] ^ A1[base + x];
                    line[x] = q[k];
                    line[x + n0] = q[k];
                }
            }
            __syncwarp();
            for (int r = 0; r < R; ++r) {
                unsigned int c = 0;
#pragma unroll
                for (int k = 0; k < kC4FastMaxL / 32; ++k)
                    if (k * 32 < n0)
                        c += __popc(q[k] ^ line[lane + 32 * k + r]);
                const unsigned int tot = __reduce_add_sync(0xffffffffu, c);
                if (lane == 0)
                    s_acc[warp][r] += tot;
            }
        }
    } else if (d == 1) {
        // a tile of 32 x-columns at one z': rows y' = 0..n1-1, doubled
        const int tiles = (n0 / 32) * N2;
        if ((int)blockIdx.x < tiles) {
            const int x0 = (blockIdx.x % (n0 / 32)) * 32, z = blockIdx.x / (n0 / 32);
            for (int y = warp; y < n1; y += 8) {
                const int w = x0 + lane + n0 * (y + n1 * z);
                const uint32_t v = A0[w] ^ A1[w];
                s_buf[y * 33 + lane] = v;
                s_buf[(y + n1) * 33 + lane] = v;
            }
            __syncthreads();
            for (int cx = warp * 4; cx < warp * 4 + 4; ++cx) {
                uint32_t q[kC4FastMaxL / 32];
#pragma unroll
                for (int k = 0; k < kC4FastMaxL / 32; ++k)
                    q[k] = k * 32 < n1 ? s_buf[(lane + 32 * k) * 33 + cx] : 0u;
                for (int r = 0; r < R; ++r) {
                    unsigned int c = 0;
#pragma unroll
                    for (int k = 0; k < kC4FastMaxL / 32; ++k)
                        if (k * 32 < n1)
                            c += __popc(q[k] ^ s_buf[(lane + 32 * k + r) * 33 + cx]);
                    const unsigned int tot = __reduce_add_sync(0xffffffffu, c);
                    if (lane == 0)
                        s_acc[warp][r] += tot;
                }
            }
        }
    } else {
        // a column (x', y') per thread, its N2 words in registers
        const int cols = n0 * n1;
        const int col = blockIdx.x * blockDim.x + threadIdx.x;
        if ((int)(blockIdx.x * blockDim.x) < cols) {
            const bool act = col < cols;
            uint32_t q[N2];
#pragma unroll
            for (int z = 0; z < N2; ++z) {
                const int w = (act ? col : 0) + n0 * n1 * z;
                q[z] = act ? (A0[w] ^ A1[w]) : 0u;
            }
            for (int r0 = 0; r0 < R; r0 += N2) {
                const int A = r0 / N2;
#pragma unroll
                for (int B = 0; B < N2; ++B) {
                    if (r0 + B >= R)
                        break;
                    unsigned int c = 0;
#pragma unroll
                    for (int z = 0; z < N2; ++z) {
                        const uint32_t p = z + B < N2 ? __funnelshift_r(q[z + B], q[z + B], A)
                                                      : __funnelshift_r(q[z + B - N2],
                                                                        q[z + B - N2], A + 1);
                        c += __popc(q[z] ^ p);
                    }
                    const unsigned int tot = __reduce_add_sync(0xffffffffu, c);
                    if (lane == 0)
                        s_acc[warp][r0 + B] += tot;
                }
            }
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w)
            t += s_acc[w][r];
        if (t)
            atomicAdd(&g_pop[((size_t)s * 3 + d) * R + r], t);
    }
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
cudaError_t launch_init_couplings(uint32_t *J, const Geo &g, int first_sample, int n_samples,
                                  double p_neg, uint64_t seed, cudaStream_t stream)
{
    const uint64_t thr_p =
        p_neg >= 1.0 ? ((uint64_t)1 << 32) : (uint64_t)floor(ldexp(p_neg, 32));
    init_couplings_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(
        J, g, thr_p, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)first_sample);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init_couplings_exact(uint32_t *J, const Geo &g, int first_sample,
                                        int n_samples, double p_neg, uint64_t seed,
                                        uint32_t *scratch, cudaStream_t stream)
{
    const uint64_t N = (uint64_t)g.L * g.L * g.L;
    const uint64_t K = (uint64_t)std::floor(p_neg * 3.0 * (double)N + 0.5);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t *state = scratch;                          // [S][4]
    uint32_t *hist = scratch + (size_t)n_samples * 4;  // [S][256]
    // prefix 0, rank K; histograms zero
    std::vector<uint32_t> init((size_t)n_samples * 4, 0u);
    for (int s = 0; s < n_samples; ++s)
        init[(size_t)s * 4 + 3] = (uint32_t)K;
    cudaError_t err = cudaMemcpyAsync(state, init.data(), init.size() * sizeof(uint32_t),
                                      cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(hist, 0, (size_t)n_samples * 256 * sizeof(uint32_t), stream);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(stream);  // init is host memory that goes away
    if (err != cudaSuccess)
        return err;
    if (K > 0) {
        const uint64_t per = (3 * N + kBlock - 1) / kBlock;
        const dim3 gh((unsigned)std::min<uint64_t>(per, 512), (unsigned)n_samples);
        for (int pass = 0; pass < 12; ++pass) {
            exact_hist_kernel<<<gh, kBlock, 0, stream>>>(g.L, pass, state, hist, k0, k1,
                                                         (uint32_t)first_sample);
            exact_select_kernel<<<n_samples, 256, 0, stream>>>(pass, state, hist);
        }
        count_launches(24);
    }
    exact_mark_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(J, g, state, K == 0 ? 1 : 0,
                                                                      k0, k1,
                                                                      (uint32_t)first_sample);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(uint32_t *spins, const Geo &g, int first_sample, int n_samples,
                              uint64_t seed, cudaStream_t stream)
{
    init_spins_kernel<<<grid_for(g, n_samples), kBlock, 0, stream>>>(
        spins, g, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)first_sample);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_obs_time(const ObsTimeParams &p, const Geo &g, int n_samples,
                            cudaStream_t stream)
{
    const unsigned bx = (unsigned)std::max(1, (g.words + 4 * kObsThreads - 1) / (4 * kObsThreads));
    obs_time_kernel<<<dim3(bx, (unsigned)n_samples), kObsThreads, 0, stream>>>(p, g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_obs_c4(const uint32_t *spins, const Geo &g, int n_samples,
                          unsigned long long *g_pop, cudaStream_t stream)
{
    if (g.k[0] == 1 && g.k[1] == 1 && g.k[2] == 32 && (g.L == 64 || g.L == 128)) {
        const int n2 = g.L / 32;
        const unsigned bx = (unsigned)std::max({g.L * n2 / 8, (g.L / 32) * n2, g.L * g.L / 256});
        const dim3 grid(bx, 3u, (unsigned)n_samples);
        if (n2 == 2)
            obs_c4_fast_kernel<2><<<grid, 256, 0, stream>>>(spins, g, g_pop);
        else
            obs_c4_fast_kernel<4><<<grid, 256, 0, stream>>>(spins, g, g_pop);
        count_launches(1);
        return cudaGetLastError();
    }
    // a block stages up to kC4Words words of whole lines of one axis
    unsigned bx = 1;
    for (int d = 0; d < 3; ++d) {
        const int lpb = kC4Words / g.n[d] > 0 ? kC4Words / g.n[d] : 1;
        const int lines = g.words / g.n[d];
        const unsigned b = (unsigned)((lines + lpb - 1) / lpb);
        bx = b > bx ? b : bx;
    }
    const dim3 grid(bx, 3u, (unsigned)n_samples);
    obs_c4_kernel<<<grid, 256, 0, stream>>>(spins, g, g_pop);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ea
