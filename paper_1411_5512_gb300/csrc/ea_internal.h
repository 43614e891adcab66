// ea_internal.h -- types shared by the library's translation units (not part
// of the public ABI).
//
// Device data layout of one job (all 32-bit words, one word = up to 32 sites
// of ONE sample, see Geo):
//   spins  [S][2][words]   "area" h of sample s holds, at word-site w, replica
//                          (h XOR colour(w)).  Half-step h updates area h and
//                          reads its neighbours from area 1-h: the interlaced
//                          checkerboard of Sec. III / Fig. 1, where one memory
//                          area holds the updated sites of both replicas.
//   J      [S][3][words]   bit = 1 <=> J = -1 for the bond from each site to its
//                          +e_d neighbour (three stored bonds per site, Sec. III).
//   snaps  [n_tw][S][2][words]  copies of spins at the waiting times.
// Bit conventions: spin bit 1 <=> S = -1; an unsatisfied bond (J S_i S_j = -1)
// is spin_i XOR spin_j XOR J = 1.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ea {

constexpr int kMaxL = 1024;
constexpr int kMaxSamples = 65535;
constexpr int kMaxSchedule = 4096;
constexpr uint64_t kMaxTime = (uint64_t)1 << 48;

// Word-site geometry: the lattice is cut into kx*ky*kz blocks of even side
// (Lx, Ly, Lz) = (L/kx, L/ky, L/kz); bit b = bx + kx*(by + ky*bz) of the word at
// word-site (x', y', z') is the site (bx*Lx + x', by*Ly + y', bz*Lz + z').
struct Geo {
    int L;
    int k[3];      // blocks per axis (powers of two)
    int n[3];      // word-lattice extent per axis (L / k)
    int stride[3]; // bit stride of an axis inside the word: 1, kx, kx*ky
    int lanes;     // kx*ky*kz
    int words;     // n[0]*n[1]*n[2]
    uint32_t valid;
    // Realignment of a neighbour word read across the periodic wrap of axis d:
    // out = ((w >> sA) & mA) | ((w << sB) & mB); index 0 for the +1 neighbour,
    // 1 for the -1 neighbour.
    uint32_t mA[3][2], mB[3][2];
    int sA[3][2], sB[3][2];
};

int make_geo(int L, Geo *g);  // 0 or -1

// Threshold planes for the bit-sliced comparison r < thr (MSB first).
struct Thr {
    uint64_t thr_u[7];      // indexed by u = number of unsatisfied bonds = 6 - k
    uint32_t always_u;      // bit u set: accepted without a random number
    uint32_t zero_calls;    // bit c set: planes 4c..4c+3 of every needed threshold are 0
    int rule;               // 0 Metropolis, 1 heat bath
    int all_always;         // every u always accepted (Metropolis at T = inf)
    int none_random;        // no lane ever needs a random number
};

struct SweepLaunch {
    uint32_t *spins;       // [S][2][words]
    const uint32_t *J;     // [S][3][words]
    Geo geo;
    Thr thr;
    uint32_t key0, key1;   // Philox key = seed
    int n_samples;
    int rng_group;         // G
};

// kernels (ea_kernels.cu); all enqueue on `stream` and return cudaGetLastError()
cudaError_t launch_init_couplings(uint32_t *J, const Geo &g, int n_samples, double p_neg,
                                  uint64_t seed, cudaStream_t stream);
cudaError_t launch_init_spins(uint32_t *spins, const Geo &g, int n_samples, uint64_t seed,
                              cudaStream_t stream);
cudaError_t launch_sweeps(const SweepLaunch &p, uint64_t t0, uint64_t n, cudaStream_t stream);

// observable sums (popcounts) accumulated with integer atomics
cudaError_t launch_obs_state(const uint32_t *spins, const uint32_t *J, const Geo &g, int n_samples,
                             unsigned long long *q_pop /*[S]*/, unsigned long long *u_pop /*[S][2]*/,
                             cudaStream_t stream);
cudaError_t launch_obs_autocorr(const uint32_t *snap, const uint32_t *spins, const Geo &g,
                                int n_samples, unsigned long long *a_pop /*[S][2]*/,
                                cudaStream_t stream);
cudaError_t launch_obs_c4(const uint32_t *spins, const Geo &g, int n_samples,
                          unsigned long long *g_pop /*[S][3][L/2+1]*/, cudaStream_t stream);

}  // namespace ea
