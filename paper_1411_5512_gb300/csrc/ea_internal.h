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

// C[g] = floor(2^64 (1 - (1 - p)^g)), g = 0..32, clamped to 2^64 - 1 (0 < p < 1).
int geo_table(double p, uint64_t C[33]);

// Acceptance tables of a job.  Both rules decide the classes u = 0, 1, 2
// (dE = 12, 8, 4) by geometric gaps with table C_u; the heat bath decides the
// classes 6 - u (dE = -12, -8, -4) with the same table, selecting the lanes
// that keep their spin, and dE = 0 by a coin word.
struct Thr {
    uint64_t geoC[3][33];   // C_u[g] = floor(2^64 (1 - (1 - p_u)^g))
    uint32_t geo_live;      // bit u: class u has a table (p_u > 0)
    uint32_t always_u;      // Metropolis, bit u set: accepted without a random number
    int rule;               // 0 Metropolis, 1 heat bath
    int all_always;         // every u always accepted (Metropolis at T = inf)
    int none_random;        // no lane ever needs a random number
};

// One job as the sweep kernel sees it (device memory).  A launch covers a
// table of jobs; block b works for the job j with block_begin[j] <= b <
// block_begin[j+1].  The plain path launches a one-entry table per job, the
// batched path one table for all jobs of a batch.
struct alignas(16) JobDev {
    uint32_t *spins;          // [S][2][words]
    const uint32_t *J;        // [S][3][words]
    uint64_t t;               // sweep index of the next sweep
    uint64_t t_end;           // the job sweeps while t < t_end (its own stop)
    Geo geo;
    uint32_t rk[20];          // Philox round keys: rk[2r], rk[2r+1] for round r
    uint32_t gC_hi[3][33];    // geometric-gap tables C_u[g], high words
    uint32_t gC_lo[3][33];    //   and low words, u = 0, 1, 2 (dE = 12, 8, 4)
    uint32_t geo_live;        // bit u: class u has a table (0 < p_u < 1)
    uint32_t always_u;        // bit u: accepted without a random number
    int rule;
    int all_always;
    int none_random;
    int n_samples;
    uint32_t rng_group;       // G
    int cols;                 // word columns per sample, n[0] * n[1]
    uint32_t div_n0_magic;    // fast division by n[0] (col -> x', y')
    int div_n0_shift;
    int blocks_per_sample;
    int cols_per_thread;
    int first_sample;         // the job-local index of the context's sample 0
    int resident;             // Metropolis: run every sweep of a launch out of shared
                              // memory, one block per sample (res_side_fits)
    int variant;              // bit 0: Metropolis side 128 on the staged kernel
    int row_lo, row_hi;       // sides 64 and 128: the rows [row_lo, row_hi) of the word
                              // lattice that sweeps update (ea_set_row_range)
    int pad_[3];
};

static_assert(sizeof(JobDev) % 16 == 0, "JobDev tables are arrays of 16-byte aligned rows");

// Host-side preparation of a JobDev (ea_sweep.cu).
void fill_job_keys(JobDev *jd, uint64_t seed);
void fill_job_thresholds(JobDev *jd, const Thr &thr);
void fill_job_layout(JobDev *jd, int cols_per_thread);

constexpr int kSweepThreads = 128;

// What the Metropolis sweep kernel reads on every word, passed in the launch's
// parameter block: indexed by a block-uniform job number, it goes through the
// uniform datapath and costs no per-thread registers.  Jobs of one side share
// a geometry record; a job record is 32 bytes, so one launch holds hundreds
// of jobs.
struct MetroGeo {
    int n0, n1, n2, cols;
    int bps, cpt;          // blocks per sample, word columns per thread
    int seg;               // rows per thread of the tile kernels
    int row0;              // the first row the tile kernels update (sides 64, 128)
    int row_n;             // and how many: threads past them update nothing
    uint32_t words;        // words per area
    uint32_t valid, magic;
    int dshift;
    uint32_t fix;          // bit 0: lanes realign across the x wrap, bit 1: y wrap
    int zsA[2], zsB[2];    // lane realignment across the periodic wrap along z
    uint32_t zmA[2], zmB[2];
    int ysA[2], ysB[2];    // and along y
    uint32_t ymA[2], ymB[2];
};

struct MetroJob {
    uint32_t *spins;
    const uint32_t *J;
    uint32_t key0, key1;   // Philox key (the seed); round keys are derived per block
    uint32_t rng_group;
    uint32_t meta;         // bits 0-2 live classes, 3 all_always, 4 none_random, 8-15 geometry,
                           // 16-31 the job-local index of the context's sample 0
};

constexpr int kMetroMaxGeo = 8;
constexpr int kMetroMaxJobs = 768;  // jobs per launch (parameter block <= 32 KB)

// A launch's job table, sized for at most MAXJ jobs; a launch takes the
// smallest size that holds its jobs, so small tables do not pay for copying a
// large parameter block.
template <int MAXJ>
struct MetroParams {
    const JobDev *jobs_dev;  // the same jobs' device rows: t, t_end, tables
    int n_jobs;
    int h;
    uint32_t sweep_offset;
    uint32_t wait_limit;     // polls of a bounded barrier wait before it gives up
    uint32_t wait_mode;      // bit 0: wait on a barrier nothing completes (tests)
    MetroGeo geo[kMetroMaxGeo];
    int block_begin[MAXJ + 1];
    MetroJob job[MAXJ];
};

static_assert(sizeof(MetroParams<kMetroMaxJobs>) <= 32000, "kernel parameter block limit");

// Kernel launches issued by the library (process-wide).  A launch made while
// the calling thread captures a graph is counted into that capture instead;
// capture_begin/capture_end bracket it and give the number of kernels the
// graph holds, which a replay adds with count_launches.
void count_launches(uint64_t n);
void capture_begin();
uint64_t capture_end();
uint64_t launches_total();

// Two side streams and the events that fork them from a launching stream and
// join them back: independent runs of a table then share the GPU.
// Sides whose half-steps take the general tiles (both rules): every lane
// along y and z (L divisible by 16), enough tiles per sample to fill a block
// (L >= 32), and not the sides with their own tile kernels (64, 128).
inline bool general_tile_side(int L)
{
    return L % 16 == 0 && L >= 32 && L != 64 && L != 128;
}

// Sides whose Metropolis samples fit whole in one block's shared memory (the
// sample-resident kernel): both spin areas, the three coupling arrays and a
// queue of one entry per word, at most kResMaxL.
constexpr int kResMaxL = 64;
inline bool res_side_fits(int L)
{
    return L >= 2 && L <= kResMaxL;
}
// The default limit: up to side 32 one block per sample is faster than a launch
// per half-step; at 48 and 64 the per-half-step kernels win unless the samples
// are few (the autotuner tries both).
constexpr int kResDefaultMaxL = 32;
// The bounded waits of the staged kernel: polls before giving up, and (tests
// of the timeout path only) a mode in which the wait is on a barrier that no
// copy completes.  Process-wide; applies to launches enqueued afterwards.
void set_wait_policy(uint32_t limit, uint32_t mode);
// Read and clear the device status word (bit 0: a bounded wait ran out),
// after the work on `stream` has finished.
cudaError_t read_sweep_status(cudaStream_t stream, uint32_t *status);

// Opt the sample-resident kernel into its shared memory (above the default
// 48 KB) on the current device; done when a context that may use it is
// created, outside any stream capture.
cudaError_t prepare_resident_kernels();
// Sweeps per launch of the sample-resident kernel (a longer request takes
// several launches), so no single launch runs for long.
constexpr uint64_t kResSweepsPerLaunch = 1024;

constexpr int kSideStreams = 4;
// Streams a batch spreads a one-kernel table over unless told otherwise: on the
// five side-128 jobs of 16 samples, 3 streams ran 18% faster than one launch
// per half-step for all of them, 2 streams 13%, 5 streams 4%.
constexpr int kDefaultStreams = 3;
struct SideStreams {
    cudaStream_t stream[kSideStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kSideStreams];
};

// Enqueue n sweeps of every job of a table: one launch per half-step per rule
// and run (tables of more than kMetroMaxJobs jobs take several).  host0/dev0
// are the host and device copies of the Metropolis rows, host1/dev1 those of
// the heat-bath rows.
// half = 0 or 1: only that half-step of one sweep (n must be 1), for a
// lattice split over ranks whose halo rows are exchanged between half-steps.
// Given side streams, the runs (the rows of one kernel) are spread over
// `stream` and the side streams, after the largest runs are halved (whole
// jobs) until there are `streams` runs (1 .. 1 + kSideStreams) or none splits.
cudaError_t launch_sweep_table(const JobDev *host0, const JobDev *dev0, int n_jobs0,
                               const JobDev *host1, const JobDev *dev1, int n_jobs1,
                               uint64_t n, cudaStream_t stream,
                               unsigned long long *counters = nullptr,
                               const SideStreams *side = nullptr, int half = -1,
                               int streams = 1);

// Four-point sums over every displacement vector (ea_c4full.cu), by an exact
// transform modulo a prime p = cL + 1 > 2N + 1 below 2^31.
constexpr int kC4FullMaxL = 512;
struct C4FullTables {
    uint32_t p;     // the prime
    uint32_t pneg;  // -p^-1 mod 2^32 (Montgomery reduction)
    uint32_t ninv;  // N^-1, Montgomery form
    uint32_t pad;
    uint32_t w[kC4FullMaxL];  // w^j, j < L, Montgomery form (w of order L, or its inverse)
};
int make_c4full_plan(int L, C4FullTables *fwd, C4FullTables *inv);  // 0 or -1
size_t c4full_scratch_words(int L);  // per sample
// Samples s0 .. s0 + n_chunk - 1 of a snapshot [S][2][words]: adds G(v) of each
// into bins[s][r^2] (zeroed by the caller), with scratch of n_chunk * L^3 words.
cudaError_t launch_c4full(const uint32_t *snap, const Geo &g, int s0, int n_chunk,
                          uint32_t *scratch, const C4FullTables &fwd, const C4FullTables &inv,
                          long long *bins, int n_bins, cudaStream_t stream);
// The static scratch of ea_c4_radial_noalloc on the current device: room for
// the bins and the residues of one sample of side up to kC4FullNoAllocMaxL.
constexpr int kC4FullNoAllocMaxL = 128;
cudaError_t c4full_static_scratch(long long **bins, uint32_t **residues);

// The integer throughput of the current device (ea_probe.cu): out[0] lop3.b32
// thread-ops/s, out[1] mad.lo.u32 thread-ops/s, out[2] Philox4x32-10 calls/s.
cudaError_t probe_int_throughput(cudaStream_t stream, double out[3]);

// Add n to the time field of every job of a table, stopping at its t_end
// (device side, for graphs).
cudaError_t launch_advance_time(JobDev *jobs_dev, int n_jobs, uint64_t n, cudaStream_t stream);

// kernels (ea_kernels.cu); all enqueue on `stream` and return cudaGetLastError()
// Samples first_sample .. first_sample + n_samples - 1 of a job: the context's
// sample s draws as the job's sample first_sample + s.
cudaError_t launch_init_couplings(uint32_t *J, const Geo &g, int first_sample, int n_samples,
                                  double p_neg, uint64_t seed, cudaStream_t stream);
// Couplings with exactly floor(p_neg 3N + 1/2) negative bonds per sample (the
// K-subset uniform); scratch holds n_samples * 260 words.
cudaError_t launch_init_couplings_exact(uint32_t *J, const Geo &g, int first_sample,
                                        int n_samples, double p_neg, uint64_t seed,
                                        uint32_t *scratch, cudaStream_t stream);
cudaError_t launch_init_spins(uint32_t *spins, const Geo &g, int first_sample, int n_samples,
                              uint64_t seed, cudaStream_t stream);

// observable sums (popcounts) accumulated with integer atomics
// The observables of one measurement time (ea_kernels.cu: obs_time_kernel):
// the state sums and the comparisons with up to kObsMaxSnaps snapshots.
constexpr int kObsMaxSnaps = 16;
constexpr int kObsThreads = 256;
struct ObsTimeParams {
    const uint32_t *spins;     // [S][2][words]
    const uint32_t *J;         // [S][3][words]
    unsigned long long *q_pop; // [S] (NULL: no state sums in this launch)
    unsigned long long *u_pop; // [S][2]
    int n_snap;
    const uint32_t *snap[kObsMaxSnaps];       // snapshots, [S][2][words] each
    unsigned long long *a_pop[kObsMaxSnaps];  // [S][2] each
};
cudaError_t launch_obs_time(const ObsTimeParams &p, const Geo &g, int n_samples,
                            cudaStream_t stream);
cudaError_t launch_obs_c4(const uint32_t *spins, const Geo &g, int n_samples,
                          unsigned long long *g_pop /*[S][3][L/2+1]*/, cudaStream_t stream);

}  // namespace ea
