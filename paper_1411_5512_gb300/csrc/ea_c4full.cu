// ea_c4full.cu -- four-point sums over every displacement vector (Eq. 3 with
// i + r any site at vector distance r from i), binned by the squared length of
// the vector's shortest periodic image: the larger point set that Sec. IV fits
// beside the axis points to size its error bars.
//
// G(v) = sum_i q_i q_{i+v} over all v in Z_L^3 is the cyclic autocorrelation
// of the q field (q_i = S^0_i S^1_i = +-1).  With Q(k) = sum_n q_n w^(n.k),
// where w has order L, sum_v G(v) w^(v.k) = Q(k) Q(-k), so
// G = DFT^-1[Q(k) Q(-k)].  The transform is taken in the integers modulo a
// prime p = cL + 1 > 2N + 1, where an element of order L exists: every step
// is exact, and G, |G| <= N, is read back from its residue.  No rounding
// enters, so the sums are bit-identical to the direct definition.
//
// The three axes are transformed in turn, each as a direct length-L DFT of
// the lines along that axis held in shared memory (any even L up to
// kC4FullMaxL).  Arithmetic is in Montgomery form with R = 2^32 (p < 2^31).
// Scratch: one uint32 residue per site and sample of a chunk of samples.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ea_internal.h"

namespace ea {
namespace {

constexpr int kLines = 32;       // lines per block of an axis pass
constexpr int kThreads = 128;
constexpr int kLoadRows = 8;     // rows per block of the first pass

__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t b, uint32_t p, uint32_t pneg)
{
    // a b R^-1 mod p for a, b < p < 2^31: t + m p < 2^62 + 2^63
    const uint64_t t = (uint64_t)a * b;
    const uint32_t m = (uint32_t)t * pneg;
    const uint32_t u = (uint32_t)((t + (uint64_t)m * p) >> 32);
    return u >= p ? u - p : u;
}

__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b, uint32_t p)
{
    const uint32_t s = a + b;  // < 2^32 for a, b < p < 2^31
    return s >= p ? s - p : s;
}

__device__ __forceinline__ uint32_t msub(uint32_t a, uint32_t b, uint32_t p)
{
    return a >= b ? a - b : a + (p - b);
}

// q bit (1 <=> q = -1) of site (x, y, z) of a sample whose two areas start at
// a0 and a0 + words: the areas hold the two replicas at every word-site.
__device__ __forceinline__ uint32_t q_bit(const uint32_t *__restrict__ a0, const Geo &g, int x,
                                          int y, int z)
{
    const int xw = x % g.n[0], yw = y % g.n[1], zw = z % g.n[2];
    const int lane = x / g.n[0] + g.k[0] * (y / g.n[1] + g.k[1] * (z / g.n[2]));
    const int w = xw + g.n[0] * (yw + g.n[1] * zw);
    return ((a0[w] ^ a0[g.words + w]) >> lane) & 1u;
}

// Pass 1: forward DFT along x of the +-1 field, read from the snapshot.  Block
// (row block, sample of the chunk); a row is (y, z).
__global__ void __launch_bounds__(kThreads)
    c4f_load_x_kernel(const uint32_t *__restrict__ snap, Geo g, int s0,
                      uint32_t *__restrict__ R, const __grid_constant__ C4FullTables tw)
{
    extern __shared__ uint32_t sm[];
    const int L = g.L;
    const int wpr = (L + 31) / 32;          // bit words per row
    uint32_t *sw = sm;                      // [L] twiddles
    uint32_t *sbits = sm + L;               // [kLoadRows][wpr]
    const int c = blockIdx.y;
    const uint32_t *a0 = snap + (size_t)(s0 + c) * 2 * g.words;
    const size_t N = (size_t)L * L * L;
    uint32_t *Rs = R + (size_t)c * N;
    const int rows = L * L;
    const int row0 = blockIdx.x * kLoadRows;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        sw[i] = tw.w[i];
    for (int i = threadIdx.x; i < kLoadRows * wpr; i += blockDim.x)
        sbits[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < kLoadRows * L; i += blockDim.x) {
        const int r = i / L, x = i - r * L, row = row0 + r;
        if (row < rows) {
            const uint32_t b = q_bit(a0, g, x, row % L, row / L);
            if (b)
                atomicOr(&sbits[r * wpr + (x >> 5)], 1u << (x & 31));
        }
    }
    __syncthreads();
    const uint32_t p = tw.p;
    for (int o = threadIdx.x; o < kLoadRows * L; o += blockDim.x) {
        const int r = o / L, k = o - r * L, row = row0 + r;
        if (row >= rows)
            continue;
        uint32_t acc = 0u;
        int idx = 0;  // x k mod L
        for (int x = 0; x < L; ++x) {
            const uint32_t v = sw[idx];
            const bool neg = ((sbits[r * wpr + (x >> 5)] >> (x & 31)) & 1u) != 0u;
            acc = madd(acc, neg ? p - v : v, p);
            idx += k;
            if (idx >= L)
                idx -= L;
        }
        Rs[(size_t)row * L + k] = acc;
    }
}

// Power-of-two sides: the +-1 field itself in Montgomery form (one = R mod p),
// for the transform pass along x that follows.
__global__ void c4f_expand_kernel(const uint32_t *__restrict__ snap, Geo g, int s0,
                                  uint32_t *__restrict__ R, uint32_t one, uint32_t p)
{
    const int L = g.L;
    const int lg = __ffs(L) - 1;  // L = 2^lg here, N < 2^31
    const uint32_t N = (uint32_t)L * L * L;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N)
        return;
    const int c = blockIdx.y;
    const uint32_t *a0 = snap + (size_t)(s0 + c) * 2 * g.words;
    const int x = (int)(i & (L - 1)), y = (int)((i >> lg) & (L - 1)), z = (int)(i >> (2 * lg));
    // the word-site and lane of (x, y, z): every extent here is a power of two
    const int sx = __ffs(g.n[0]) - 1, sy = __ffs(g.n[1]) - 1, sz = __ffs(g.n[2]) - 1;
    const int kx = __ffs(g.k[0]) - 1, ky = __ffs(g.k[1]) - 1;
    const int w = (x & (g.n[0] - 1)) | ((y & (g.n[1] - 1)) << sx) | ((z & (g.n[2] - 1)) << (sx + sy));
    const int lane = (x >> sx) | ((y >> sy) << kx) | ((z >> sz) << (kx + ky));
    const uint32_t b = ((a0[w] ^ a0[g.words + w]) >> lane) & 1u;
    R[(size_t)c * N + i] = b ? p - one : one;
}

// Address of element e of line g along an axis (0 x, 1 y, 2 z) of one sample.
__device__ __forceinline__ size_t line_addr(int axis, int L, int g, int e)
{
    if (axis == 0)
        return (size_t)g * L + e;
    const int x = g % L, o = g / L;
    if (axis == 1)
        return (size_t)x + (size_t)L * e + (size_t)L * L * o;
    return (size_t)x + (size_t)L * o + (size_t)L * L * e;
}

// A DFT pass along one axis, in place, for kLines lines per block.  With bins
// (the last inverse pass, along x) the results are read out of Montgomery
// form and added into the radial bins of the sample instead of written back.
// With RADIX2 (L a power of two) the lines are transformed in place by the
// iterative radix-2 scheme: elements loaded in bit-reversed order, log2 L
// stages of butterflies (u, v w) -> (u + v w, u - v w) with w = w^(j L / len),
// the result in natural order; O is then T itself.
template <bool BIN, bool RADIX2>
__global__ void __launch_bounds__(kThreads)
    c4f_axis_kernel(uint32_t *__restrict__ R, int L, int axis,
                    const __grid_constant__ C4FullTables tw, long long *__restrict__ bins,
                    int n_bins, int s0)
{
    extern __shared__ uint32_t sm[];
    constexpr int P = kLines + 1;  // tile pitch
    uint32_t *sw = sm;             // [L]
    uint32_t *T = sm + L;          // [L][P] input
    uint32_t *O = RADIX2 ? T : T + L * P;  // [L][P] output
    const int c = blockIdx.y;
    const size_t N = (size_t)L * L * L;
    uint32_t *Rs = R + (size_t)c * N;
    const int lines = L * L;
    const int g0 = blockIdx.x * kLines;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        sw[i] = tw.w[i];
    // load: along x the elements of a line are contiguous, along y and z the
    // lines of a block are (mostly) adjacent in x
    for (int i = threadIdx.x; i < kLines * L; i += blockDim.x) {
        int l, e;
        if (axis == 0) {
            l = i / L;
            e = i - l * L;
        } else {
            e = i / kLines;
            l = i - e * kLines;
        }
        const int g = g0 + l;
        int et = e;
        if (RADIX2)
            et = (int)(__brev((uint32_t)e) >> (32 - (__ffs(L) - 1)));
        T[et * P + l] = g < lines ? Rs[line_addr(axis, L, g, e)] : 0u;
    }
    __syncthreads();
    const uint32_t p = tw.p, pneg = tw.pneg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (RADIX2) {
        for (int len = 2; len <= L; len <<= 1) {
            const int half = len >> 1, step = L / len;
            for (int k = warp; k < L / 2; k += kThreads / 32) {
                const int j = k & (half - 1);
                const int i0 = (k - j) * 2 + j, i1 = i0 + half;
                const uint32_t u = T[i0 * P + lane];
                const uint32_t v = mmul(T[i1 * P + lane], sw[j * step], p, pneg);
                T[i0 * P + lane] = madd(u, v, p);
                T[i1 * P + lane] = msub(u, v, p);
            }
            __syncthreads();
        }
    } else {
        for (int k = warp; k < L; k += kThreads / 32) {
            uint32_t acc = 0u;
            int idx = 0;  // e k mod L
            for (int e = 0; e < L; ++e) {
                acc = madd(acc, mmul(T[e * P + lane], sw[idx], p, pneg), p);
                idx += k;
                if (idx >= L)
                    idx -= L;
            }
            O[k * P + lane] = acc;
        }
        __syncthreads();
    }
    if (!BIN) {
        for (int i = threadIdx.x; i < kLines * L; i += blockDim.x) {
            int l, e;
            if (axis == 0) {
                l = i / L;
                e = i - l * L;
            } else {
                e = i / kLines;
                l = i - e * kLines;
            }
            const int g = g0 + l;
            if (g < lines)
                Rs[line_addr(axis, L, g, e)] = O[e * P + l];
        }
        return;
    }
    // the last pass runs along x: line g is the row (dy, dz) = (g mod L, g / L);
    // G(dx) and G(L - dx) share the bin m^2 + my^2 + mz^2 with m = min(dx, L - dx)
    const int H = L / 2;
    long long *bs = bins + (size_t)(s0 + c) * n_bins;
    for (int i = threadIdx.x; i < kLines * (H + 1); i += blockDim.x) {
        const int l = i / (H + 1), m = i - l * (H + 1);
        const int g = g0 + l;
        if (g >= lines)
            continue;
        const int dy = g % L, dz = g / L;
        const int my = min(dy, L - dy), mz = min(dz, L - dz);
        long long v = 0;
        for (int side = 0; side < 2; ++side) {
            const int dx = side == 0 ? m : L - m;
            if (side == 1 && (m == 0 || m == H))
                break;
            const uint32_t r = mmul(O[dx * P + l], 1u, p, pneg);  // out of Montgomery form
            v += r > (p >> 1) ? (long long)r - (long long)p : (long long)r;
        }
        atomicAdd(reinterpret_cast<unsigned long long *>(bs + m * m + my * my + mz * mz),
                  (unsigned long long)v);
    }
}

// Q(k) Q(-k) N^-1, written to both k and -k.
__global__ void c4f_pointwise_kernel(uint32_t *__restrict__ R, int L, uint32_t p, uint32_t pneg,
                                     uint32_t ninv)
{
    const size_t N = (size_t)L * L * L;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N)
        return;
    uint32_t *Rs = R + (size_t)blockIdx.y * N;
    const int kx = (int)(i % L), ky = (int)((i / L) % L), kz = (int)(i / ((size_t)L * L));
    const int jx = kx == 0 ? 0 : L - kx, jy = ky == 0 ? 0 : L - ky, jz = kz == 0 ? 0 : L - kz;
    const size_t j = (size_t)jx + (size_t)L * (jy + (size_t)L * jz);
    if (i > j)
        return;  // the pair is handled by its lower index
    const uint32_t v = mmul(mmul(Rs[i], Rs[j], p, pneg), ninv, p, pneg);
    Rs[i] = v;
    Rs[j] = v;
}

size_t axis_smem(int L, bool radix2)
{
    return ((size_t)L + (radix2 ? 1 : 2) * (size_t)L * (kLines + 1)) * sizeof(uint32_t);
}

bool is_prime(uint32_t n)
{
    if (n < 2)
        return false;
    for (uint32_t d = 2; (uint64_t)d * d <= n; ++d)
        if (n % d == 0)
            return false;
    return true;
}

uint32_t pow_mod(uint32_t b, uint64_t e, uint32_t p)
{
    uint64_t r = 1, x = b % p;
    while (e) {
        if (e & 1)
            r = r * x % p;
        x = x * x % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

uint32_t to_mont(uint32_t x, uint32_t p)
{
    return (uint32_t)((((uint64_t)x) << 32) % p);
}

}  // namespace

int make_c4full_plan(int L, C4FullTables *fwd, C4FullTables *inv)
{
    if (L < 2 || (L & 1) || L > kC4FullMaxL)
        return -1;
    const uint64_t N = (uint64_t)L * L * L;
    // the smallest prime p = cL + 1 above 2N + 1
    uint64_t p = 0;
    for (uint64_t c = (2 * N + 2) / L + 1;; ++c) {
        p = c * L + 1;
        if (p >= ((uint64_t)1 << 31))
            return -1;
        if (is_prime((uint32_t)p))
            break;
    }
    const uint32_t P = (uint32_t)p;
    // a generator of the multiplicative group: g^((p-1)/q) != 1 for each prime
    // q | p - 1 (fewer than 10 distinct ones below 2^31)
    uint32_t qs[32];
    int nq = 0;
    uint32_t m = P - 1;
    for (uint32_t d = 2; (uint64_t)d * d <= m; ++d)
        if (m % d == 0) {
            qs[nq++] = d;
            while (m % d == 0)
                m /= d;
        }
    if (m > 1)
        qs[nq++] = m;
    uint32_t gen = 2;
    for (;; ++gen) {
        bool ok = true;
        for (int i = 0; i < nq; ++i)
            ok = ok && pow_mod(gen, (P - 1) / qs[i], P) != 1u;
        if (ok)
            break;
    }
    const uint32_t w = pow_mod(gen, (P - 1) / (uint32_t)L, P);  // order L
    const uint32_t wi = pow_mod(w, (uint64_t)L - 1, P);
    uint32_t pinv = P;  // p^-1 mod 2^32 by Newton's iteration (p odd)
    for (int i = 0; i < 5; ++i)
        pinv *= 2u - P * pinv;
    std::memset(fwd, 0, sizeof(*fwd));
    std::memset(inv, 0, sizeof(*inv));
    fwd->p = inv->p = P;
    fwd->pneg = inv->pneg = 0u - pinv;
    fwd->ninv = inv->ninv = to_mont(pow_mod((uint32_t)(N % P), P - 2, P), P);
    uint64_t a = 1, b = 1;
    for (int j = 0; j < L; ++j) {
        fwd->w[j] = to_mont((uint32_t)a, P);
        inv->w[j] = to_mont((uint32_t)b, P);
        a = a * w % P;
        b = b * wi % P;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Scratch without allocation, for ea_c4_radial_noalloc: some callers cannot
// call cudaMalloc (a host that has handed all device memory to its own pool,
// or code on a path where an allocation, which may synchronise the device, is
// not allowed).  They get the transform's scratch from this file-scope array:
// the radial bins of one sample, then the residues of one sample of side up
// to kC4FullNoAllocMaxL.  Every process that loads the library holds it on
// every device it uses, until exit.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocBinsU64 = 12320;  // 3 (128/2)^2 + 1 = 12289 bins, padded to 256 bytes
constexpr size_t kNoAllocU64 =
    kNoAllocBinsU64 + (size_t)kC4FullNoAllocMaxL * kC4FullNoAllocMaxL * kC4FullNoAllocMaxL / 2;
static __device__ __align__(256) unsigned long long g_c4full_scratch[kNoAllocU64];

cudaError_t c4full_static_scratch(long long **bins, uint32_t **residues)
{
    // the array's device address, looked up once per device with that device
    // current (in host code the array's name is only a stand-in)
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static void *addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess)
        return err;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_c4full_scratch);
        if (err != cudaSuccess)
            return err;
        addr[dev] = p;
    }
    unsigned long long *base = static_cast<unsigned long long *>(addr[dev]);
    *bins = reinterpret_cast<long long *>(base);
    *residues = reinterpret_cast<uint32_t *>(base + kNoAllocBinsU64);
    return cudaSuccess;
}

size_t c4full_scratch_words(int L)
{
    return (size_t)L * L * L;
}

template <bool RADIX2>
cudaError_t launch_c4full_passes(const uint32_t *snap, const Geo &g, int s0, int n_chunk,
                                 uint32_t *scratch, const C4FullTables &fwd,
                                 const C4FullTables &inv, long long *bins, int n_bins,
                                 cudaStream_t stream)
{
    const int L = g.L;
    const size_t sm = axis_smem(L, RADIX2);
    cudaError_t err = cudaFuncSetAttribute(c4f_axis_kernel<false, RADIX2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(c4f_axis_kernel<true, RADIX2>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess)
        return err;
    const int lines = L * L;
    const size_t N = (size_t)L * L * L;
    const dim3 g_axis((lines + kLines - 1) / kLines, n_chunk);
    int launches = 0;
    if (RADIX2) {
        // the +-1 field, then its transform along x
        const dim3 g_ex((unsigned)((N + 255) / 256), n_chunk);
        c4f_expand_kernel<<<g_ex, 256, 0, stream>>>(snap, g, s0, scratch,
                                                    (uint32_t)(((uint64_t)1 << 32) % fwd.p),
                                                    fwd.p);
        c4f_axis_kernel<false, RADIX2>
            <<<g_axis, kThreads, sm, stream>>>(scratch, L, 0, fwd, nullptr, 0, s0);
        launches += 2;
    } else {
        const dim3 g_load((lines + kLoadRows - 1) / kLoadRows, n_chunk);
        const size_t sm_load =
            ((size_t)L + kLoadRows * (size_t)((L + 31) / 32)) * sizeof(uint32_t);
        c4f_load_x_kernel<<<g_load, kThreads, sm_load, stream>>>(snap, g, s0, scratch, fwd);
        launches += 1;
    }
    c4f_axis_kernel<false, RADIX2><<<g_axis, kThreads, sm, stream>>>(scratch, L, 1, fwd, nullptr, 0,
                                                                     s0);
    c4f_axis_kernel<false, RADIX2><<<g_axis, kThreads, sm, stream>>>(scratch, L, 2, fwd, nullptr, 0,
                                                                     s0);
    const dim3 g_pw((unsigned)((N + 255) / 256), n_chunk);
    c4f_pointwise_kernel<<<g_pw, 256, 0, stream>>>(scratch, L, fwd.p, fwd.pneg, fwd.ninv);
    c4f_axis_kernel<false, RADIX2><<<g_axis, kThreads, sm, stream>>>(scratch, L, 2, inv, nullptr, 0,
                                                                     s0);
    c4f_axis_kernel<false, RADIX2><<<g_axis, kThreads, sm, stream>>>(scratch, L, 1, inv, nullptr, 0,
                                                                     s0);
    c4f_axis_kernel<true, RADIX2><<<g_axis, kThreads, sm, stream>>>(scratch, L, 0, inv, bins,
                                                                    n_bins, s0);
    count_launches((uint64_t)launches + 6);
    return cudaGetLastError();
}

cudaError_t launch_c4full(const uint32_t *snap, const Geo &g, int s0, int n_chunk,
                          uint32_t *scratch, const C4FullTables &fwd, const C4FullTables &inv,
                          long long *bins, int n_bins, cudaStream_t stream)
{
    // power-of-two sides by the radix-2 transform, the others by direct DFTs
    if ((g.L & (g.L - 1)) == 0)
        return launch_c4full_passes<true>(snap, g, s0, n_chunk, scratch, fwd, inv, bins, n_bins,
                                          stream);
    return launch_c4full_passes<false>(snap, g, s0, n_chunk, scratch, fwd, inv, bins, n_bins,
                                       stream);
}

}  // namespace ea
