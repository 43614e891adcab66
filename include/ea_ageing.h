/*
 * ea_ageing.h -- C ABI of the GB300 (sm_103a) library for the non-equilibrium
 * ageing simulation of the three-dimensional +-J Edwards-Anderson model of
 * Manssen & Hartmann, "Ageing at the Spin-Glass/Ferromagnet Transition: Monte
 * Carlo Simulation using GPUs" (arXiv 1411.5512).
 *
 * One context ("job") holds n_samples disorder samples of an L^3 periodic
 * lattice, each with two replicas that share the couplings (Sec. II, Eq. 2),
 * quenched from a random start (Sec. II) and evolved by single-spin-flip
 * Metropolis sweeps in checkerboard order (Sec. III, Eq. 9), or by the
 * heat-bath rule.  Measurements of the autocorrelation C(t, t_w) (Eq. 7), the
 * replica overlap q (Eq. 2), the four-point correlation C4(r, t_w) (Eq. 3)
 * along the lattice axes and the integral estimator xi_1 (Eqs. 5-6) are taken
 * on the device at the times of a schedule; C4 over every displacement vector
 * is computed on request from the snapshots (ea_c4_radial).
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: EA_OK (0) or a negative EA_ERR_*.
 *     No call aborts the process or throws across the ABI.  After an error on
 *     a context, ea_last_error(ctx) describes it.
 *   - Host pointers are plain C arrays owned by the caller; the library never
 *     keeps them after the call returns.  Device memory is owned by the context
 *     and released by ea_destroy.
 *   - p_neg is the fraction of NEGATIVE (antiferromagnetic) couplings, i.e.
 *     1 - p in the paper's P(J) = p delta(J - 1) + (1 - p) delta(J + 1)
 *     (Sec. II).  p_neg = 0.5 is the spin glass, p_neg = 0 the ferromagnet.
 *   - Spins are reported as int8 +-1 in the order [z][y][x] (x fastest); the
 *     coupling array J[d][z][y][x] (d = x, y, z) holds the bond between a site
 *     and its +e_d neighbour, with periodic boundaries (Sec. II).
 *   - L must be even (a checkerboard on a periodic lattice), 2 <= L <= 1024.
 *   - Sweep t (t = 0, 1, ...) updates, in half-step h = 0 then h = 1, every
 *     site of colour (x + y + z) mod 2 == h XOR a of replica a, so replica 1
 *     runs the opposite colour order (the interlaced layout of Fig. 1).  After
 *     n sweeps the context time is n; measurements at time m see the state
 *     after m sweeps.
 *   - Results are bit-identical to the CPU oracle on the same arguments.
 *     The random numbers are keyed by (seed, sample div G, word-site,
 *     replica, sweep) and by the energy class and draw index inside a
 *     word-site, never by where a job runs: a word-site groups up to 32 sites
 *     of one sample (ea_geometry), and the sites of one energy class in a
 *     word-site are decided together by geometric gaps, so the decision of a
 *     site depends on which other lanes of its word-site share its class.
 *     Each site still flips independently with its probability of Eq. 9.
 */
#ifndef EA_AGEING_H
#define EA_AGEING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define EA_OK 0
#define EA_ERR_INVALID_ARG (-1) /* argument out of range (odd L, p outside [0,1], ...) */
#define EA_ERR_OOM (-2)         /* device or host allocation failed */
#define EA_ERR_NO_SNAPSHOT (-3) /* (t_w, t) not scheduled or not reached yet */
#define EA_ERR_STATE (-4)       /* call out of order (e.g. sweep before quench) */
#define EA_ERR_TIMEOUT (-5)     /* a bounded device wait ran out */
#define EA_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define EA_ERR_IO (-7)          /* checkpoint file could not be written or read */

/* ---- update rules ------------------------------------------------------- */
#define EA_RULE_METROPOLIS 0 /* p = min(1, exp(-dE/T))      (Sec. III, Eq. 9) */
#define EA_RULE_HEATBATH 1   /* p = 1 / (1 + exp(dE/T))     (variant)         */

typedef struct ea_ctx ea_ctx;

/* Observables of one (t_w, t) pair, filled by ea_measure.  Every array pointer
 * may be NULL (then it is skipped); non-NULL arrays are caller-owned host
 * memory of the stated sizes.  S = n_samples, R = L/2 + 1. */
typedef struct ea_obs {
    int64_t *A;      /* [S][2]  sum_i S_i(t_w) S_i(t_w + t) per replica     (Eq. 7 x N) */
    int64_t *Q;      /* [S]     sum_i S^0_i S^1_i at time t_w + t          (Eq. 2 x N) */
    int64_t *E;      /* [S][2]  H = -sum_<ij> J_ij S_i S_j at t_w + t       (Eq. 1)     */
    int64_t *G;      /* [S][3][R] sum_i q_i q_{i + r e_d}, d = x,y,z, at t_w (Eq. 3 x N) */
    double *C4;      /* [R]     C4(r, t_w), averaged over axes and samples            */
    double *C4_sem;  /* [R]     standard error of C4 over samples (NaN if S < 2)       */
    double C;        /* C(t, t_w), averaged over replicas and samples     (Eq. 7)     */
    double q_mean;   /* sample mean of q at time t_w + t                  (Eq. 2)     */
    double xi1;      /* xi_1(t_w) = I_2 / I_1 over r = 1..r_cut (Eqs. 5-6); NaN if empty */
    int r_cut;       /* last r before C4 first drops below 3 * C4_sem (L/2 if never)   */
} ea_obs;

/* ---- host-only helpers (no GPU needed) ---------------------------------- */

/* Human-readable name of a status code.  Never NULL. */
const char *ea_status_string(int status);

/* Geometry of the random-number mapping for lattice side L (Sec. III's
 * multi-part packing, over three axes): out = {kx, ky, kz, L/kx, L/ky, L/kz}.
 * The lattice is cut into kx*ky*kz <= 32 blocks of even side and the sites at
 * the same position in every block form one 32-bit word.  Rule: h = L/2,
 * p2 = largest power of two dividing h, kz = min(32, p2), ky = min(32/kz, p2),
 * kx = min(32/(kz*ky), p2).  EA_ERR_INVALID_ARG for odd L or L outside [2,1024]. */
int ea_geometry(int L, int out[6]);

/* Flip probabilities for dE = 4k - 12, k = 0..6, as 64-bit fixed point:
 * thr[k] = floor(2^64 P(dE)), where P is min(1, exp(-dE/T)) for
 * EA_RULE_METROPOLIS (Eq. 9) and 1/(1 + exp(dE/T)) for EA_RULE_HEATBATH;
 * P = 1 sets always[k] (and thr[k] = 0).  T = 0 and T = +inf give the limits.
 * The sweeps realise these probabilities class by class: the sites of a
 * word-site with one dE are decided by geometric gaps (ea_geo_table; for the
 * heat bath with dE < 0 the gaps select the sites that keep their spin), and
 * the heat bath's dE = 0 sites by a fair coin.  Both arrays are caller-owned.
 * EA_ERR_INVALID_ARG for T < 0, NaN T or an unknown rule. */
int ea_thresholds(double T, int rule, uint64_t thr[7], uint8_t always[7]);

/* Geometric-gap table of the updates: C[g] = floor(2^64 (1 - (1 - p)^g)) for
 * g = 0..32 (clamped to 2^64 - 1), computed as floor(ldexp(-expm1(g
 * log1p(-p)), 64)).  Among the n sites of one word-site with the same dE > 0,
 * each selected independently with probability p (Metropolis: the flip
 * probability exp(-dE/T), Eq. 9; heat bath: 1/(1 + exp(dE/T)), which also
 * selects the sites that keep their spin at -dE), a 64-bit uniform V selects
 * none when V >= C[n], else the site of rank min{g : V < C[g+1]} in increasing
 * lane order; the sites after it start a fresh gap with the next draw.
 * EA_ERR_INVALID_ARG unless 0 < p < 1.  Host-only. */
int ea_geo_table(double p, uint64_t C[33]);

/* Device bytes a context with this shape and schedule will hold (spins,
 * couplings, snapshots and results).  Host-only arithmetic. */
int ea_footprint(int L, int n_samples, int n_tw, int n_t, size_t *bytes);

/* ---- device memory hook -------------------------------------------------- */

/* Route the library's device allocations through the caller (for example a
 * framework's caching allocator).  alloc(bytes, stream, user) returns a device
 * pointer or NULL; release(ptr, bytes, stream, user) frees it.  Passing NULL
 * for both restores cudaMalloc / cudaFree.  Process-wide; call it while no
 * context exists. */
typedef void *(*ea_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*ea_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int ea_set_allocator(ea_alloc_fn alloc, ea_free_fn release, void *user);

/* ---- launch accounting --------------------------------------------------- */

/* Number of kernel launches the library has issued in this process: every
 * direct launch, plus the kernels of a captured CUDA graph each time the graph
 * is replayed (capturing itself counts nothing).  Thread-safe; never fails.
 * The difference across a region of host code counts the library's kernels
 * enqueued in it. */
uint64_t ea_launch_count(void);

/* The integer throughput of the current device, measured by three short
 * kernels of independent dependency chains that fill every SM: out[0] =
 * three-input logic ops (lop3.b32) per second, out[1] = 32-bit multiply-adds
 * (mad.lo.u32) per second, out[2] = Philox4x32-10 calls per second, each the
 * best of five timed launches.  The paper has no counterpart: these are the
 * denominators of the integer-ALU roofline that the sweep is reported
 * against.  Allocates nothing; synchronises the stream.  Errors:
 * EA_ERR_INVALID_ARG (NULL out), EA_ERR_CUDA. */
int ea_int_throughput(void *cuda_stream, double out[3]);

/* Bounded waits on the device.  Every wait of a kernel on a barrier (the
 * staged kernel waits for its bulk copies) polls at most `polls` times; when a
 * wait runs out, the block waits for its own copies still in flight, sets
 * bit 0 of the device status word and returns, leaving its rows of that
 * half-step unfinished, so the context stays usable and the host learns of it
 * from ea_device_status.  The default is 2^22 polls.  wait_for_nothing = 1 is
 * for tests of that path only: the waits are then on a barrier that no copy
 * ever completes, so each runs out after `polls` polls.  Process-wide; applies
 * to launches enqueued afterwards.  Errors: EA_ERR_INVALID_ARG
 * (wait_for_nothing not 0 or 1). */
int ea_debug_set_wait(uint32_t polls, int wait_for_nothing);

/* Synchronises the stream, reads and clears the device status word: *status
 * bit 0 = a bounded wait ran out since the last read.  Returns EA_ERR_TIMEOUT
 * when bit 0 is set, EA_ERR_CUDA when the read fails, else EA_OK. */
int ea_device_status(void *cuda_stream, uint32_t *status);

/* ---- job lifecycle ------------------------------------------------------- */

/* Create a job of n_samples samples of side L and generate their couplings on
 * the device: J = -1 with probability p_neg, independently per bond (Sec. II,
 * Eq. 1's bimodal P(J)).  rng_group_G >= 1 samples share each sweep random
 * number (the paper shares one number across the samples of a word, Sec. III;
 * G = 1 gives every sample its own); disorder and start stay per sample.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream); every device
 * call of the job is enqueued on it.  *out receives the new context.
 * Errors: EA_ERR_INVALID_ARG (odd L, L out of range, p_neg outside [0,1],
 * n_samples < 1, G < 1), EA_ERR_OOM, EA_ERR_CUDA. */
int ea_create_samples(ea_ctx **out, int L, double p_neg, uint64_t seed, int n_samples,
                      int rng_group_G, void *cuda_stream);

/* As ea_create_samples, but every sample has exactly K = floor(p_neg 3N + 1/2)
 * negative bonds, the K-subset uniform among all of them, instead of
 * independent bonds.  Sec. II draws every bond independently from P(J); this
 * variant fixes the concentration of each sample instead, which removes its
 * sample-to-sample fluctuation.  Bond b = d N + i (d = x, y, z; i the site) gets the 64-bit key
 * (out0 << 32) | out1 of Philox4x32-10 with counter (i, 1 + d, 0, s) and key
 * (lo32(seed), hi32(seed)); the negative bonds are the first K in the order
 * of (key, b).  Synchronises the stream.  Errors as ea_create_samples. */
int ea_create_samples_exact(ea_ctx **out, int L, double p_neg, uint64_t seed, int n_samples,
                            int rng_group_G, void *cuda_stream);

/* Samples first_sample .. first_sample + n_samples - 1 of the job
 * (L, p_neg, seed, G): the context's sample s is the job's sample
 * first_sample + s, with that index in every random number (couplings,
 * initial spins, sweeps; its share group is (first_sample + s) div G).  So
 * disjoint ranges of one job, run in different processes or on different
 * GPUs, give bit for bit the samples that ea_create_samples would give for the
 * whole job, and their integer sums add up to the whole job's (Sec. III: the
 * paper ran independent sample batches on each GPU).  ea_create_samples is
 * the range starting at 0.  Errors as ea_create_samples, and
 * EA_ERR_INVALID_ARG for first_sample < 0 or first_sample + n_samples above
 * 65535. */
int ea_create_samples_range(ea_ctx **out, int L, double p_neg, uint64_t seed, int first_sample,
                            int n_samples, int rng_group_G, void *cuda_stream);

/* Set the measurement schedule: waiting times t_w[0..n_tw) and time lags
 * t[0..n_t) (Sec. II: C(t, t_w) and C4(r, t_w) are measured at waiting times
 * counted in sweeps from the quench).  At every t_w the state is snapshotted
 * and Q, E and the four-point sums G are taken; at every t_w + t the
 * autocorrelation against the t_w snapshot and Q, E are taken.  Duplicates
 * are ignored.  Must precede ea_quench.  Arrays are caller-owned.
 * Errors: EA_ERR_INVALID_ARG (n < 0, more than 4096 entries, time >= 2^48),
 * EA_ERR_STATE (after quench), EA_ERR_OOM. */
int ea_set_schedule(ea_ctx *ctx, const uint64_t *t_w, int n_tw, const uint64_t *t, int n_t);

/* Quench: draw uniform random initial spins for both replicas of every
 * sample (Sec. II, start from infinite temperature), set the thresholds for
 * temperature T and the update rule, reset the time to 0 and take the time-0
 * measurements of the schedule.  May be called again to restart.
 * Errors: EA_ERR_INVALID_ARG (T < 0, NaN, unknown rule), EA_ERR_CUDA. */
int ea_quench(ea_ctx *ctx, double T, int rule);

/* Run n sweeps (Sec. III: one sweep = both checkerboard half-steps), firing
 * the scheduled snapshots and measurements on the way.  Asynchronous: work is
 * enqueued on the job's stream.  Errors: EA_ERR_STATE (before ea_quench),
 * EA_ERR_INVALID_ARG (time would pass 2^48), EA_ERR_CUDA. */
int ea_sweep(ea_ctx *ctx, uint64_t n);

/* One lattice split over ranks (y-slabs, the single-lattice decomposition
 * over several GPUs that Sec. III sketches for lattices larger than one
 * GPU).  Sides 64 and 128, whose word lattice has every lane along z, so that
 * a row y' of the word lattice is the lattice row y:
 *   ea_set_row_range: sweeps of this context update only the rows [y_lo,
 *     y_hi); the other rows are read as neighbours and must be kept current
 *     by the caller.  Needs a context with no measurement schedule that is not
 *     in a batch (EA_ERR_STATE).  EA_ERR_INVALID_ARG for other sides or rows.
 *     Not saved by ea_checkpoint.
 *   ea_half_sweep: the next half-step of the current sweep (h = 0, then
 *     h = 1, after which the time advances by one), so that the halo rows can
 *     be exchanged between the two.  Needs a context with no schedule.
 *   ea_get_rows / ea_set_rows: rows y .. y + n_rows - 1 of spin area `area`
 *     (0 or 1: half-step h updates area h and reads area 1 - h) of every
 *     sample, to or from host words laid out [sample][z'][row][x'];
 *     synchronises the stream.
 * A rank owning rows [lo, hi) sends its rows lo and hi - 1 of area 1 - h
 * before half-step h and receives rows lo - 1 and hi (periodic); the result
 * is bit-identical to the undivided lattice. */
int ea_set_row_range(ea_ctx *ctx, int y_lo, int y_hi);
int ea_half_sweep(ea_ctx *ctx);
int ea_get_rows(ea_ctx *ctx, int area, int y, int n_rows, uint32_t *host_words);
int ea_set_rows(ea_ctx *ctx, int area, int y, int n_rows, const uint32_t *host_words);

/* Current time (sweeps done since the quench, counting sweeps still enqueued)
 * into *t.  Host only.  Errors: EA_ERR_INVALID_ARG (NULL). */
int ea_time(const ea_ctx *ctx, uint64_t *t);

/* Read back the observables of the pair (t_w, t) into *out and derive the
 * FP64 quantities (C, q, C4, its error, r_cut, xi_1; Eqs. 2, 3, 5-7).
 * Synchronises the job's stream.  Errors: EA_ERR_NO_SNAPSHOT when t_w is not
 * a scheduled waiting time, t not a scheduled lag, or t_w + t not reached. */
int ea_measure(ea_ctx *ctx, uint64_t t_w, uint64_t t, ea_obs *out);

/* Four-point sums over every displacement vector, binned by distance (Eq. 3
 * with i + r any site at vector distance r from i; Sec. IV fits this larger
 * point set beside the axis points to size its error bars).
 * For the snapshot at the scheduled waiting time t_w and every sample s:
 *   sums[s * n_bins + b] = sum over vectors v with |v|^2 = b of
 *                          sum_i q_i q_{i+v},   q_i = S^0_i S^1_i,
 * where |v|^2 = sum over axes of min(d, L - d)^2 (the shortest periodic
 * image), b = 0 .. n_bins - 1, and counts[b] = the number of vectors with
 * |v|^2 = b (0 for the values no vector takes).  Exact integers: computed by
 * a transform modulo a prime, with no rounding.  The caller owns
 * sums[n_samples * n_bins] and counts[n_bins] (n_bins from
 * ea_c4_radial_bins).  The FP64 curve goes to C4[n_bins] and
 * C4_sem[n_bins] when they are not NULL: for a bin b with counts[b] > 0,
 *   C4[b]     = sum_s sums[s][b] / (counts[b] N n_samples)  (one rounding),
 *   C4_sem[b] = the standard error over samples of sums[s][b] / (counts[b] N)
 *               (NaN with one sample);
 * both NaN where counts[b] = 0.  Uses device scratch of up to 256 MiB while
 * it runs and synchronises the job's stream.  Errors: EA_ERR_INVALID_ARG
 * (NULL sums or counts, side above 512), EA_ERR_STATE (before ea_quench),
 * EA_ERR_NO_SNAPSHOT (t_w not scheduled or not reached), EA_ERR_OOM. */
int ea_c4_radial(ea_ctx *ctx, uint64_t t_w, long long *sums, long long *counts, double *C4,
                 double *C4_sem);

/* ea_c4_radial for callers that cannot allocate device memory: a host that
 * has handed all of it to its own pool, or code on a path where cudaMalloc,
 * which may synchronise the device, is not allowed.  The paper has no
 * counterpart; this is a property of the library.  Same arguments, results
 * and errors as ea_c4_radial, but it calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch is a static device array built into the
 * library, room for one sample of side up to 128 (8.1 MiB, held on every
 * device the process uses, until exit).  Samples go through it one at a time.
 * Sides above 128 give EA_ERR_INVALID_ARG.  The first call on a device looks
 * up the array's address on that device (make it before any stream capture),
 * with the job's device current.  All calls share the array and it keeps the
 * last call's contents (each call clears what it sums into first): calls that
 * overlap on the GPU, from different streams or threads, race, so order them.
 * Synchronises the job's stream. */
int ea_c4_radial_noalloc(ea_ctx *ctx, uint64_t t_w, long long *sums, long long *counts,
                         double *C4, double *C4_sem);

/* Number of distance bins of ea_c4_radial for side L: 3 (L/2)^2 + 1.
 * Host only.  EA_ERR_INVALID_ARG for odd L, L < 2 or L > 512. */
int ea_c4_radial_bins(int L, int *n_bins);

/* Copy spins of sample s, replica a into out[L^3] (int8 +-1, [z][y][x]).
 * Synchronous.  Errors: EA_ERR_INVALID_ARG, EA_ERR_STATE (before quench). */
int ea_get_spins(ea_ctx *ctx, int s, int a, int8_t *out);

/* Copy couplings of sample s into out[3][L^3] (int8 +-1, [d][z][y][x]; J[d] is
 * the bond to the +e_d neighbour).  Valid from ea_create_samples on.
 * Synchronous.  Errors: EA_ERR_INVALID_ARG (NULL, s out of range), EA_ERR_CUDA. */
int ea_get_couplings(ea_ctx *ctx, int s, int8_t *out);

/* Load a configuration (the paper stores whole configurations at its
 * measurement points, Sec. IV): replace the spins of sample s, replica a by
 * in[L^3] (int8 +-1, [z][y][x]), or its couplings by in[3][L^3] ([d][z][y][x]),
 * and set the time counter with ea_set_time (sweep t then draws the random
 * numbers of sweep t).  Snapshots and results already taken are kept.
 * Synchronous.  Errors: EA_ERR_INVALID_ARG (a value other than +-1, bad
 * index, time >= 2^48), EA_ERR_STATE (spins or time before ea_quench). */
int ea_set_spins(ea_ctx *ctx, int s, int a, const int8_t *in);
int ea_set_couplings(ea_ctx *ctx, int s, const int8_t *in);
int ea_set_time(ea_ctx *ctx, uint64_t t);

/* The couplings of every sample in the library's packed layout, moved in one
 * copy: words J[s][d][w], s < n_samples, d = x, y, z, w < words (the word
 * lattice of ea_geometry); bit b of J[s][d][w] is 1 when the bond from the
 * site at word-site w, lane b, to its +e_d neighbour is J = -1.  Lanes past
 * the word's sites (fewer than 32 lanes, small L) are 0.  n_words =
 * n_samples * 3 * words.  get copies device to host; set copies host to
 * device (bits outside the lanes: EA_ERR_INVALID_ARG) and replaces the
 * couplings drawn by ea_create_samples.  Both synchronise the job's stream;
 * pinned host memory makes the copy a single DMA. */
int ea_coupling_words(const ea_ctx *ctx, size_t *n_words);
int ea_get_coupling_words(ea_ctx *ctx, uint32_t *host_words);
int ea_set_coupling_words(ea_ctx *ctx, const uint32_t *host_words);

/* Thresholds in use (as ea_thresholds).  EA_ERR_STATE before ea_quench. */
int ea_get_thresholds(const ea_ctx *ctx, uint64_t thr[7], uint8_t always[7]);

/* Write the whole job (parameters, time, schedule, spins, couplings,
 * snapshots, results) to a file; ea_restore rebuilds it on cuda_stream.  The
 * random numbers are counter-based, so a restored job continues bit-identically.
 * Errors: EA_ERR_IO, EA_ERR_STATE (before quench), EA_ERR_CUDA, EA_ERR_OOM. */
int ea_checkpoint(ea_ctx *ctx, const char *path);
int ea_restore(ea_ctx **out, const char *path, void *cuda_stream);

/* Release the job and its device memory.  NULL is accepted. */
int ea_destroy(ea_ctx *ctx);

/* Text of the last error on ctx (empty string if none).  Never NULL. */
const char *ea_last_error(const ea_ctx *ctx);

/* ---- batching: many jobs, one launch per half-step ------------------------
 *
 * A batch sweeps many quenched jobs together: every half-step of every
 * member, whatever its L, p_neg, T, rule or sample count, is one kernel launch
 * over a table of jobs (Sec. III: one launch per half-step keeps the global
 * synchronisation of the checkerboard).  With graph_sweeps > 0 the launches of
 * graph_sweeps sweeps are captured once into a CUDA graph and replayed.  Each
 * member keeps its own time, schedule and random stream, so a job gives
 * bit-identical results alone and in any batch.
 *
 * While a job is a member, its work (sweeps and measurements) is enqueued on
 * the batch's stream; ea_measure and the other per-job calls stay valid.  The
 * batch does not own its members: remove (or destroy the batch) before
 * ea_destroy on a member. */
typedef struct ea_batch ea_batch;

/* New empty batch on cuda_stream (NULL = legacy stream; graphs then stay off).
 * Errors: EA_ERR_OOM. */
int ea_batch_create(ea_batch **out, void *cuda_stream);

/* Add / remove a quenched job.  Errors: EA_ERR_INVALID_ARG (NULL, already a
 * member / not a member), EA_ERR_STATE (job not quenched). */
int ea_batch_add(ea_batch *b, ea_ctx *job);
int ea_batch_remove(ea_batch *b, ea_ctx *job);

/* Number of member jobs into *n_jobs.  Errors: EA_ERR_INVALID_ARG (NULL). */
int ea_batch_size(const ea_batch *b, int *n_jobs);

/* Launch shape used by ea_batch_sweep: work per thread of the sweep kernel
 * (1, 2 or 4; 0 = per-job default) and sweeps per captured graph (0 = direct
 * launches).  The work per thread is that many word columns, or for a table
 * whose jobs all have side 64 or 128, segments of 4, 8 or 16 rows of 2 x 2
 * word-sites.  Neither changes any result.  get reads both back.  Errors:
 * EA_ERR_INVALID_ARG (NULL, cols_per_thread other than 0, 1, 2, 4, graph_sweeps
 * outside 0..4096). */
int ea_batch_configure(ea_batch *b, int cols_per_thread, int graph_sweeps);
int ea_batch_get_config(const ea_batch *b, int *cols_per_thread, int *graph_sweeps);

/* Metropolis members of side up to max_side (and at most 64) run sample-
 * resident: one block per sample holds the sample's spins and couplings in
 * shared memory and runs every sweep of a launch there (up to 1024), instead
 * of one launch per half-step over memory (Sec. III: each half-step its own
 * kernel with a global synchronisation between them).  0 turns it off.  The
 * results do not change.  New batches use 32, and so does a context swept on
 * its own (ea_sweep): up to side 32 one block per sample beats a launch per
 * half-step.  The autotuner chooses among 32, 64 and 0.  get reads it back.
 * Errors: EA_ERR_INVALID_ARG (NULL, max_side < 0). */
int ea_batch_set_resident(ea_batch *b, int max_side);
int ea_batch_get_resident(const ea_batch *b, int *max_side);

/* The kernel of side-128 Metropolis members: 0 (the default) the
 * register-window tile kernel; 1 the staged kernel, whose blocks bring each
 * row of the state into shared memory with bulk asynchronous copies while the
 * previous row is computed.  Both give the same results; the staged
 * kernel applies when the tables of dE = 8 and 12 are small (T below about
 * 1), the tile kernel otherwise.  The autotuner also chooses between them.
 * Errors: EA_ERR_INVALID_ARG (NULL, variant not 0 or 1). */
int ea_batch_set_variant(ea_batch *b, int variant);
int ea_batch_get_variant(const ea_batch *b, int *variant);

/* The streams a batch spreads its sweep launches over, 1 .. 5 (default 3).
 * The members form one group per kernel (side range and rule); while there
 * are fewer groups than streams, the group of most jobs is halved (whole
 * jobs).  Each group's half-step launches go to a stream of its own, forked
 * from the batch's stream and joined back after the sweeps, so one group's
 * launches fill the SMs that another group's last wave leaves idle.  Jobs are
 * independent, so the results do not depend on the setting; with 1 a
 * one-kernel batch runs one launch per half-step for all its members.  The
 * autotuner chooses among 1 .. 4.  get reads it back.
 * Errors: EA_ERR_INVALID_ARG (NULL, streams outside 1 .. 5). */
int ea_batch_set_streams(ea_batch *b, int streams);
int ea_batch_get_streams(const ea_batch *b, int *streams);

/* Try the launch configurations on the members' current state for
 * trial_sweeps sweeps each: word columns per thread {1, 2, 4}, graphs {none,
 * 16, 64 sweeps} (at most trial_sweeps), and where they apply the resident limit {32, 64, 0}, the
 * side-128 kernel {0, 1} and the streams {1, 2, 3, 4}.  Keeps the fastest and
 * puts the state back as it was (time, spins): the tuning leaves every result
 * unchanged.  Synchronises the batch stream. */
int ea_batch_autotune(ea_batch *b, int trial_sweeps);

/* Work counts of the update, for the integer-op roofline: runs `sweeps`
 * sweeps of every member with a counting variant of the sweep kernel and
 * then puts the members' state back (time, spins), so no result changes.
 * out = {word updates, Philox4x32-10 calls, the calls among them that the
 * rare path makes (extension and continuation draws, beyond the main calls),
 * attempted spin flips}.  The call count is per word with per-word early
 * exit, i.e. what the algorithm needs, not what a SIMT warp issues.
 * Synchronises the batch stream.  Errors: EA_ERR_INVALID_ARG (NULL, sweeps
 * < 1), EA_ERR_CUDA, EA_ERR_OOM. */
int ea_batch_profile(ea_batch *b, int sweeps, uint64_t out[4]);

/* Run n sweeps of every member, firing each member's scheduled measurements
 * at its own times.  Asynchronous on the batch stream.
 * Errors: EA_ERR_INVALID_ARG (a member's time would pass 2^48), EA_ERR_CUDA. */
int ea_batch_sweep(ea_batch *b, uint64_t n);

/* Destroy the batch; members return to their own streams.  NULL is accepted. */
int ea_batch_destroy(ea_batch *b);

/* Text of the last error on the batch (empty string if none or NULL); owned by
 * the batch, valid until its next call.  Never NULL. */
const char *ea_batch_last_error(const ea_batch *b);

/* ---- serving: continuous batching of ageing jobs ---------------------------
 *
 * A server keeps a queue of submitted jobs and a batch of running ones.  Each
 * ea_server_step (1) admits queued jobs in submission order that fit, by
 * device footprint (ea_footprint) within the byte budget and by the slot
 * limit, skipping ones that do not fit yet; (2) advances every running job by
 * up to chunk_sweeps sweeps in the batch's launches, each job stopping at its
 * own sweep count; (3) retires finished jobs.  Jobs that arrive while others
 * are on the GPU join at the next step, so their work overlaps on the device.
 * A job's results depend only on its own spec (seed, sample index, time),
 * never on what else ran with it.  Finished jobs keep their device memory,
 * and their budget share, until ea_server_release. */
typedef struct ea_server ea_server;

typedef struct ea_job_spec {
    int L;
    double p_neg;
    uint64_t seed;
    int n_samples;
    int rng_group_G;
    double T;
    int rule;
    uint64_t sweeps;           /* the job is done after this many sweeps */
    const uint64_t *t_w;       /* measurement schedule, as ea_set_schedule */
    int n_tw;
    const uint64_t *t;
    int n_t;
} ea_job_spec;

#define EA_JOB_QUEUED 0
#define EA_JOB_RUNNING 1
#define EA_JOB_DONE 2

typedef struct ea_server_stats {
    int queued, running, done;
    size_t bytes_in_use;       /* footprint of running and unreleased jobs */
    uint64_t flips;            /* attempted spin flips run so far */
    uint64_t steps;
} ea_server_stats;

/* New server.  budget_bytes: device bytes its jobs may hold; max_running:
 * slots; chunk_sweeps: sweeps per step (> 0).  Errors: EA_ERR_INVALID_ARG,
 * EA_ERR_OOM. */
int ea_server_create(ea_server **out, size_t budget_bytes, int max_running, uint64_t chunk_sweeps,
                     void *cuda_stream);

/* Queue a job (copies the spec and its schedule arrays).  *job_id receives
 * its id.  Errors: EA_ERR_INVALID_ARG (bad spec, or a footprint above the
 * whole budget). */
int ea_server_submit(ea_server *srv, const ea_job_spec *spec, int64_t *job_id);

/* One step: admit, run one chunk, retire.  *n_finished (may be NULL)
 * receives the number of jobs retired in this step.  Asynchronous apart from
 * the admission of new jobs; a retired job's results are read with
 * ea_measure on its context (ea_server_job), which synchronises. */
int ea_server_step(ea_server *srv, int *n_finished);

/* Launch shape of the running set, as ea_batch_configure (default: 4 word
 * columns per thread, 16-sweep graphs off the legacy stream).  No result
 * depends on it. */
int ea_server_configure(ea_server *srv, int cols_per_thread, int graph_sweeps);

/* State (EA_JOB_*) and time of a job. */
int ea_server_job_state(const ea_server *srv, int64_t job_id, int *state, uint64_t *time);

/* The job's context (owned by the server; valid until ea_server_release),
 * for ea_measure / ea_get_spins.  EA_ERR_STATE while the job is queued. */
int ea_server_job(ea_server *srv, int64_t job_id, ea_ctx **job);

/* Free a finished job's device memory and its budget share.
 * EA_ERR_STATE unless the job is done. */
int ea_server_release(ea_server *srv, int64_t job_id);

/* Cancel a queued or running job: it leaves the queue or the batch at once
 * (work already enqueued completes first) and its memory is freed.  A done
 * job is released.  EA_ERR_INVALID_ARG for an unknown id. */
int ea_server_cancel(ea_server *srv, int64_t job_id);

/* Counts of queued, running and done (unreleased) jobs, bytes in use, flips
 * and steps so far, into the caller's *out.  Host only.  Errors:
 * EA_ERR_INVALID_ARG (NULL). */
int ea_server_get_stats(const ea_server *srv, ea_server_stats *out);

/* Destroy the server and every job it still holds.  NULL is accepted. */
int ea_server_destroy(ea_server *srv);

/* Text of the last error on the server (empty string if none or NULL); owned
 * by the server, valid until its next call.  Never NULL. */
const char *ea_server_last_error(const ea_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* EA_AGEING_H */
