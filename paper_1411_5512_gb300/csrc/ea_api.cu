// ea_api.cu -- host runtime behind the C ABI of include/ea_ageing.h.
//
// A context owns the bit-packed device state of one job (couplings, both
// replicas of every sample, snapshots at the waiting times, integer result
// counters), the measurement schedule and the job's CUDA stream.  The sweep
// loop runs on the host: chunks of sweeps between scheduled measurement
// times are enqueued as half-step launches (Sec. III: one launch per
// half-step gives the global synchronisation), measurements are enqueued
// in between, and nothing synchronises until results are read back.
#include <algorithm>
#include <atomic>
#include <deque>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ea_ageing.h"
#include <nvtx3/nvToolsExt.h>

#include "ea_internal.h"

using ea::Geo;

namespace {

ea_alloc_fn g_alloc = nullptr;
ea_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;

// An NVTX range over a call that enqueues work: named spans on a profiler's
// timeline (nsys, ncu --nvtx); without a tool attached it costs a branch.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

void *dev_alloc(size_t bytes, cudaStream_t stream)
{
    if (bytes == 0)
        bytes = 16;
    if (g_alloc)
        return g_alloc(bytes, (void *)stream, g_alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t stream)
{
    if (!p)
        return;
    if (bytes == 0)
        bytes = 16;
    if (g_free)
        g_free(p, bytes, (void *)stream, g_alloc_user);
    else
        cudaFree(p);
}

}  // namespace

namespace ea {

static std::atomic<uint64_t> g_launches{0};
static thread_local bool tl_capturing = false;
static thread_local uint64_t tl_captured = 0;

void count_launches(uint64_t n)
{
    if (tl_capturing)
        tl_captured += n;
    else
        g_launches.fetch_add(n, std::memory_order_relaxed);
}

void capture_begin()
{
    tl_capturing = true;
    tl_captured = 0;
}

uint64_t capture_end()
{
    tl_capturing = false;
    return tl_captured;
}

uint64_t launches_total()
{
    return g_launches.load(std::memory_order_relaxed);
}

int make_geo(int L, Geo *g)
{
    if (L < 2 || L > kMaxL || (L & 1))
        return -1;
    std::memset(g, 0, sizeof(*g));
    const int h = L / 2;
    const int p2 = h & (-h);
    const int kz = std::min(32, p2);
    const int ky = std::min(32 / kz, p2);
    const int kx = std::min(32 / (kz * ky), p2);
    g->L = L;
    g->k[0] = kx;
    g->k[1] = ky;
    g->k[2] = kz;
    for (int d = 0; d < 3; ++d)
        g->n[d] = L / g->k[d];
    g->stride[0] = 1;
    g->stride[1] = kx;
    g->stride[2] = kx * ky;
    g->lanes = kx * ky * kz;
    g->words = g->n[0] * g->n[1] * g->n[2];
    g->valid = g->lanes == 32 ? 0xffffffffu : ((1u << g->lanes) - 1u);
    for (int d = 0; d < 3; ++d) {
        const int k = g->k[d], st = g->stride[d];
        for (int dir = 0; dir < 2; ++dir) {
            if (k == 1) {
                g->sA[d][dir] = 0;
                g->sB[d][dir] = 0;
                g->mA[d][dir] = g->valid;
                g->mB[d][dir] = 0;
                continue;
            }
            // +1 neighbour: lane with block index b reads block index b+1 (mod k);
            // -1 neighbour: b-1, i.e. a shift by k-1.
            const int q = dir == 0 ? 1 : k - 1;
            uint32_t mA = 0;
            for (int b = 0; b < g->lanes; ++b)
                if ((b / st) % k < k - q)
                    mA |= 1u << b;
            g->sA[d][dir] = q * st;
            g->sB[d][dir] = (k - q) * st;
            g->mA[d][dir] = mA;
            g->mB[d][dir] = g->valid & ~mA;
        }
    }
    return 0;
}

int geo_table(double p, uint64_t C[33])
{
    if (!(p > 0.0 && p < 1.0))
        return -1;
    C[0] = 0;
    for (int g = 1; g <= 32; ++g) {
        // 1 - (1 - p)^g, accurate for tiny p
        const double q = -std::expm1((double)g * std::log1p(-p));
        const double v = std::ldexp(q, 64);
        C[g] = v >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)std::floor(v);
    }
    return 0;
}

}  // namespace ea

// ---------------------------------------------------------------------------
// thresholds (Eq. 9 and the heat-bath rule), host FP64
// ---------------------------------------------------------------------------
static int compute_thresholds(double T, int rule, uint64_t thr[7], uint8_t always[7])
{
    if (!(T >= 0.0) || (rule != EA_RULE_METROPOLIS && rule != EA_RULE_HEATBATH))
        return EA_ERR_INVALID_ARG;
    for (int k = 0; k < 7; ++k) {
        const int dE = 4 * k - 12;
        double P;
        if (rule == EA_RULE_METROPOLIS) {
            // min(1, exp(-dE/T)); T = 0 leaves only downhill and level moves
            if (dE <= 0)
                P = 1.0;
            else if (T == 0.0)
                P = 0.0;
            else
                P = std::exp(-(double)dE / T);
        } else {
            if (T == 0.0)
                P = dE < 0 ? 1.0 : (dE == 0 ? 0.5 : 0.0);
            else
                P = 1.0 / (1.0 + std::exp((double)dE / T));
        }
        if (P >= 1.0) {
            always[k] = 1;
            thr[k] = 0;
        } else {
            always[k] = 0;
            thr[k] = (uint64_t)std::floor(std::ldexp(P, 64));
        }
    }
    return EA_OK;
}

static ea::Thr make_thr(int rule, double T, const uint64_t thr_k[7], const uint8_t always_k[7])
{
    ea::Thr t;
    std::memset(&t, 0, sizeof(t));
    t.rule = rule;
    if (rule == EA_RULE_METROPOLIS) {
        // classes u = 0, 1, 2 (dE = 12, 8, 4) decided by geometric gaps
        for (int u = 0; u < 3; ++u) {
            const int k = 6 - u;
            if (always_k[k]) {
                // accepted outright: every non-empty class hits its table and
                // the rare path flips all of its lanes
                t.geo_live |= 1u << u;
                for (int g = 1; g <= 32; ++g)
                    t.geoC[u][g] = ~(uint64_t)0;
            } else if (thr_k[k] > 0) {
                t.geo_live |= 1u << u;
                ea::geo_table(std::exp(-(double)(12 - 4 * u) / T), t.geoC[u]);
            }
        }
        int n_always = 0;
        for (int u = 0; u < 7; ++u)
            if (always_k[6 - u]) {  // u unsatisfied bonds <=> k = 6 - u
                t.always_u |= 1u << u;
                ++n_always;
            }
        t.all_always = n_always == 7;
        // no class can accept: the random numbers are skipped
        t.none_random = t.geo_live == 0;
    } else if (T > 0.0) {
        // heat bath: p_u = 1 / (1 + e^((12 - 4u)/T)) for dE = 12 - 4u > 0; the
        // table of p_u also selects the lanes of class 6 - u that keep their
        // spin.  p_u = 0 (T = 0 or beyond the double range) leaves no table.
        for (int u = 0; u < 3; ++u) {
            const double p = 1.0 / (1.0 + std::exp((double)(12 - 4 * u) / T));
            if (p > 0.0) {
                t.geo_live |= 1u << u;
                ea::geo_table(p, t.geoC[u]);
            }
        }
    }
    return t;
}

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
struct ea_ctx {
    int L = 0;
    double p_neg = 0;
    uint64_t seed = 0;
    int S = 0;
    int first = 0;  // the job-local index of sample 0 (ea_create_samples_range)
    int G = 1;
    int half = 0;   // 1 between the two half-steps of a sweep (ea_half_sweep)
    cudaStream_t stream = nullptr;
    Geo geo;

    uint32_t *spins = nullptr;
    uint32_t *J = nullptr;
    uint32_t *snaps = nullptr;
    ea::JobDev jd;                 // host copy of the job's sweep-table entry
    ea::JobDev *jd_dev = nullptr;  // one-entry table for the plain path
    unsigned long long *res = nullptr;
    size_t spins_bytes = 0, J_bytes = 0, snaps_bytes = 0, res_bytes = 0;
    // host copy of res, valid while res_gen == res_host_gen; res_gen moves on
    // whenever work that writes res is enqueued
    std::vector<unsigned long long> res_host;
    uint64_t res_gen = 1, res_host_gen = 0;

    std::vector<uint64_t> tw, tt, meas;
    size_t off_q = 0, off_u = 0, off_g = 0, off_a = 0;  // in counters

    bool quenched = false;
    double T = 0;
    int rule = 0;
    uint64_t thr_k[7] = {0};
    uint8_t always_k[7] = {0};
    ea::Thr thr;
    uint64_t t = 0;

    ea_batch *batch = nullptr;          // batch this job belongs to, if any
    cudaStream_t own_stream = nullptr;  // the job's stream outside a batch

    std::string err;

    size_t words_per_sample() const { return (size_t)geo.words; }
    size_t area_words() const { return (size_t)S * 2 * geo.words; }
    int R() const { return L / 2 + 1; }
};

namespace {

int fail(ea_ctx *c, int code, const std::string &msg)
{
    if (c)
        c->err = msg;
    return code;
}

int cuda_fail(ea_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(c, EA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define EA_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess)                               \
            return cuda_fail((ctx), e_, #call);              \
    } while (0)

void release_schedule(ea_ctx *c)
{
    dev_free(c->snaps, c->snaps_bytes, c->stream);
    dev_free(c->res, c->res_bytes, c->stream);
    c->snaps = nullptr;
    c->res = nullptr;
    c->snaps_bytes = c->res_bytes = 0;
}

int idx_of(const std::vector<uint64_t> &v, uint64_t x)
{
    auto it = std::lower_bound(v.begin(), v.end(), x);
    if (it == v.end() || *it != x)
        return -1;
    return (int)(it - v.begin());
}

std::vector<uint64_t> sorted_unique(const uint64_t *p, int n)
{
    std::vector<uint64_t> v(p, p + n);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
}

size_t results_counters(int S, int R, size_t n_meas, size_t n_tw, size_t n_t)
{
    return n_meas * (size_t)S * 3 + n_tw * (size_t)S * 3 * R + n_tw * n_t * (size_t)S * 2;
}

int build_schedule(ea_ctx *c, std::vector<uint64_t> tw, std::vector<uint64_t> tt)
{
    std::vector<uint64_t> meas = tw;
    for (uint64_t a : tw)
        for (uint64_t b : tt)
            if (a + b < ea::kMaxTime)
                meas.push_back(a + b);
    std::sort(meas.begin(), meas.end());
    meas.erase(std::unique(meas.begin(), meas.end()), meas.end());

    release_schedule(c);
    c->tw = std::move(tw);
    c->tt = std::move(tt);
    c->meas = std::move(meas);
    const size_t S = (size_t)c->S, R = (size_t)c->R();
    c->off_q = 0;
    c->off_u = c->off_q + c->meas.size() * S;
    c->off_g = c->off_u + c->meas.size() * S * 2;
    c->off_a = c->off_g + c->tw.size() * S * 3 * R;
    const size_t n_ctr = results_counters(c->S, c->R(), c->meas.size(), c->tw.size(), c->tt.size());
    c->res_bytes = n_ctr * sizeof(unsigned long long);
    ++c->res_gen;
    c->snaps_bytes = c->tw.size() * c->area_words() * sizeof(uint32_t);
    if (c->res_bytes) {
        c->res = (unsigned long long *)dev_alloc(c->res_bytes, c->stream);
        if (!c->res)
            return fail(c, EA_ERR_OOM, "results allocation failed");
    }
    if (c->snaps_bytes) {
        c->snaps = (uint32_t *)dev_alloc(c->snaps_bytes, c->stream);
        if (!c->snaps) {
            release_schedule(c);
            return fail(c, EA_ERR_OOM, "snapshot allocation failed");
        }
    }
    return EA_OK;
}

int upload_job(ea_ctx *c)
{
    c->jd.t = c->t;
    c->jd.t_end = c->t;
    EA_CUDA(c, cudaMemcpyAsync(c->jd_dev, &c->jd, sizeof(ea::JobDev), cudaMemcpyHostToDevice,
                               c->stream));
    return EA_OK;
}

// The plain path's table entry runs sweeps t .. t_end-1 of the next chunk.
int upload_time(ea_ctx *c, uint64_t t_end)
{
    static_assert(offsetof(ea::JobDev, t_end) == offsetof(ea::JobDev, t) + sizeof(uint64_t),
                  "t and t_end are uploaded together");
    c->jd.t = c->t;
    c->jd.t_end = t_end;
    EA_CUDA(c, cudaMemcpyAsync(&c->jd_dev->t, &c->jd.t, 2 * sizeof(uint64_t),
                               cudaMemcpyHostToDevice, c->stream));
    return EA_OK;
}

int launch_plain(ea_ctx *c, uint64_t n)
{
    const bool heat = c->rule == EA_RULE_HEATBATH;
    EA_CUDA(c, ea::launch_sweep_table(heat ? nullptr : &c->jd, heat ? nullptr : c->jd_dev,
                                      heat ? 0 : 1, heat ? &c->jd : nullptr,
                                      heat ? c->jd_dev : nullptr, heat ? 1 : 0, n, c->stream));
    return EA_OK;
}

// Measurements due at the current time c->t (if it is a scheduled time).
int fire_measurements(ea_ctx *c, cudaStream_t stream)
{
    const int mi = idx_of(c->meas, c->t);
    if (mi < 0)
        return EA_OK;
    ++c->res_gen;
    const size_t S = (size_t)c->S, R = (size_t)c->R();
    const size_t area = c->area_words();
    const int ti = idx_of(c->tw, c->t);
    if (ti >= 0) {
        EA_CUDA(c, cudaMemcpyAsync(c->snaps + ti * area, c->spins, area * sizeof(uint32_t),
                                   cudaMemcpyDeviceToDevice, stream));
        EA_CUDA(c, ea::launch_obs_c4(c->spins, c->geo, c->S, c->res + c->off_g + ti * S * 3 * R,
                                     stream));
    }
    // the state sums and every autocorrelation due at this time, one pass over
    // the state per launch of up to kObsMaxSnaps snapshots
    ea::ObsTimeParams p;
    std::memset(&p, 0, sizeof(p));
    p.spins = c->spins;
    p.J = c->J;
    p.q_pop = c->res + c->off_q + mi * S;
    p.u_pop = c->res + c->off_u + mi * S * 2;
    for (size_t i = 0; i < c->tw.size() && c->tw[i] <= c->t; ++i) {
        const int j = idx_of(c->tt, c->t - c->tw[i]);
        if (j < 0)
            continue;
        p.snap[p.n_snap] = c->snaps + i * area;
        p.a_pop[p.n_snap] = c->res + c->off_a + (i * c->tt.size() + (size_t)j) * S * 2;
        if (++p.n_snap == ea::kObsMaxSnaps) {
            EA_CUDA(c, ea::launch_obs_time(p, c->geo, c->S, stream));
            p.q_pop = nullptr;  // the state sums went with the first launch
            p.u_pop = nullptr;
            p.n_snap = 0;
        }
    }
    if (p.n_snap > 0 || p.q_pop != nullptr)
        EA_CUDA(c, ea::launch_obs_time(p, c->geo, c->S, stream));
    return EA_OK;
}

int check_ctx(const ea_ctx *c) { return c ? EA_OK : EA_ERR_INVALID_ARG; }

}  // namespace

// Default launch shape of the sweep kernels: enough blocks to fill the GPU a
// few times over for one job, fewer per-thread set-ups for large lattices.
// Sides 64 and 128 take their tile kernels, whose threads already hold 4 rows
// of 2 x 2 word-sites at the smallest shape.
static int default_cols_per_thread(const Geo &g)
{
    if (g.L == 64 || g.L == 128)
        return 1;
    const int cols = g.n[0] * g.n[1];
    return cols >= 8192 ? 2 : 1;
}

namespace {

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *ea_status_string(int status)
{
    switch (status) {
    case EA_OK: return "EA_OK";
    case EA_ERR_INVALID_ARG: return "EA_ERR_INVALID_ARG";
    case EA_ERR_OOM: return "EA_ERR_OOM";
    case EA_ERR_NO_SNAPSHOT: return "EA_ERR_NO_SNAPSHOT";
    case EA_ERR_STATE: return "EA_ERR_STATE";
    case EA_ERR_TIMEOUT: return "EA_ERR_TIMEOUT";
    case EA_ERR_CUDA: return "EA_ERR_CUDA";
    case EA_ERR_IO: return "EA_ERR_IO";
    default: return "EA_ERR_UNKNOWN";
    }
}

int ea_geometry(int L, int out[6])
{
    Geo g;
    if (!out || ea::make_geo(L, &g) != 0)
        return EA_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d) {
        out[d] = g.k[d];
        out[3 + d] = g.n[d];
    }
    return EA_OK;
}

int ea_thresholds(double T, int rule, uint64_t thr[7], uint8_t always[7])
{
    if (!thr || !always)
        return EA_ERR_INVALID_ARG;
    return compute_thresholds(T, rule, thr, always);
}

int ea_geo_table(double p, uint64_t C[33])
{
    if (!C)
        return EA_ERR_INVALID_ARG;
    return ea::geo_table(p, C) == 0 ? EA_OK : EA_ERR_INVALID_ARG;
}

int ea_footprint(int L, int n_samples, int n_tw, int n_t, size_t *bytes)
{
    Geo g;
    if (!bytes || ea::make_geo(L, &g) != 0 || n_samples < 1 || n_samples > ea::kMaxSamples ||
        n_tw < 0 || n_t < 0 || n_tw > ea::kMaxSchedule || n_t > ea::kMaxSchedule)
        return EA_ERR_INVALID_ARG;
    const size_t W = (size_t)g.words * n_samples * sizeof(uint32_t);
    const size_t n_meas = (size_t)n_tw + (size_t)n_tw * n_t;  // upper bound
    *bytes = W * 2 + W * 3 + (size_t)n_tw * W * 2 +
             results_counters(n_samples, L / 2 + 1, n_meas, n_tw, n_t) * 8;
    return EA_OK;
}

int ea_debug_set_wait(uint32_t polls, int wait_for_nothing)
{
    if (wait_for_nothing != 0 && wait_for_nothing != 1)
        return EA_ERR_INVALID_ARG;
    ea::set_wait_policy(polls, (uint32_t)wait_for_nothing);
    return EA_OK;
}

int ea_device_status(void *cuda_stream, uint32_t *status)
{
    if (!status)
        return EA_ERR_INVALID_ARG;
    if (ea::read_sweep_status((cudaStream_t)cuda_stream, status) != cudaSuccess) {
        cudaGetLastError();
        return EA_ERR_CUDA;
    }
    return (*status & 1u) ? EA_ERR_TIMEOUT : EA_OK;
}

int ea_int_throughput(void *cuda_stream, double out[3])
{
    if (!out)
        return EA_ERR_INVALID_ARG;
    if (ea::probe_int_throughput((cudaStream_t)cuda_stream, out) != cudaSuccess) {
        cudaGetLastError();
        return EA_ERR_CUDA;
    }
    return EA_OK;
}

int ea_set_allocator(ea_alloc_fn alloc, ea_free_fn release, void *user)
{
    if ((alloc == nullptr) != (release == nullptr))
        return EA_ERR_INVALID_ARG;
    g_alloc = alloc;
    g_free = release;
    g_alloc_user = user;
    return EA_OK;
}

int ea_create_samples(ea_ctx **out, int L, double p_neg, uint64_t seed, int n_samples,
                      int rng_group_G, void *cuda_stream)
{
    return ea_create_samples_range(out, L, p_neg, seed, 0, n_samples, rng_group_G, cuda_stream);
}

int ea_create_samples_range(ea_ctx **out, int L, double p_neg, uint64_t seed, int first_sample,
                            int n_samples, int rng_group_G, void *cuda_stream)
{
    NvtxRange nvtx_range("ea_create_samples");
    if (!out)
        return EA_ERR_INVALID_ARG;
    *out = nullptr;
    Geo g;
    if (ea::make_geo(L, &g) != 0 || !(p_neg >= 0.0 && p_neg <= 1.0) || n_samples < 1 ||
        first_sample < 0 || n_samples > ea::kMaxSamples - first_sample || rng_group_G < 1)
        return EA_ERR_INVALID_ARG;
    ea_ctx *c = new (std::nothrow) ea_ctx();
    if (!c)
        return EA_ERR_OOM;
    c->L = L;
    c->p_neg = p_neg;
    c->seed = seed;
    c->S = n_samples;
    c->first = first_sample;
    c->G = rng_group_G;
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = c->stream;
    c->geo = g;
    c->spins_bytes = c->area_words() * sizeof(uint32_t);
    c->J_bytes = (size_t)n_samples * 3 * g.words * sizeof(uint32_t);
    c->spins = (uint32_t *)dev_alloc(c->spins_bytes, c->stream);
    c->J = (uint32_t *)dev_alloc(c->J_bytes, c->stream);
    c->jd_dev = (ea::JobDev *)dev_alloc(sizeof(ea::JobDev), c->stream);
    if (!c->spins || !c->J || !c->jd_dev) {
        ea_destroy(c);
        return EA_ERR_OOM;
    }
    std::memset(&c->jd, 0, sizeof(c->jd));
    c->jd.spins = c->spins;
    c->jd.J = c->J;
    c->jd.geo = g;
    c->jd.n_samples = n_samples;
    c->jd.first_sample = first_sample;
    c->jd.row_lo = 0;
    c->jd.row_hi = g.n[1];
    c->jd.resident = L <= ea::kResDefaultMaxL && ea::res_side_fits(L) ? 1 : 0;
    c->jd.variant = 0;  // side 128: the register-window tile kernel
    if (c->jd.resident) {
        // the kernel's shared-memory opt-in, per device, outside any capture
        int dev = 0;
        static std::mutex mu;
        static std::vector<int> ready;
        std::lock_guard<std::mutex> lock(mu);
        if (cudaGetDevice(&dev) == cudaSuccess &&
            std::find(ready.begin(), ready.end(), dev) == ready.end()) {
            if (ea::prepare_resident_kernels() != cudaSuccess) {
                cudaGetLastError();
                ea_destroy(c);
                return EA_ERR_CUDA;
            }
            ready.push_back(dev);
        }
    }
    c->jd.rng_group = (uint32_t)rng_group_G;
    ea::fill_job_keys(&c->jd, seed);
    ea::fill_job_layout(&c->jd, default_cols_per_thread(g));
    cudaError_t e =
        ea::launch_init_couplings(c->J, g, first_sample, n_samples, p_neg, seed, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->spins, 0, c->spins_bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ea_destroy(c);
        return EA_ERR_CUDA;
    }
    *out = c;
    return EA_OK;
}

int ea_create_samples_exact(ea_ctx **out, int L, double p_neg, uint64_t seed, int n_samples,
                            int rng_group_G, void *cuda_stream)
{
    const int rc = ea_create_samples(out, L, p_neg, seed, n_samples, rng_group_G, cuda_stream);
    if (rc != EA_OK)
        return rc;
    ea_ctx *c = *out;
    // the i.i.d. couplings just drawn are replaced by the exact-count draw
    const size_t scratch_bytes = (size_t)n_samples * 260 * sizeof(uint32_t);
    uint32_t *scratch = (uint32_t *)dev_alloc(scratch_bytes, c->stream);
    if (!scratch) {
        ea_destroy(c);
        *out = nullptr;
        return EA_ERR_OOM;
    }
    cudaError_t e = ea::launch_init_couplings_exact(c->J, c->geo, c->first, n_samples, p_neg,
                                                    seed, scratch, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    dev_free(scratch, scratch_bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ea_destroy(c);
        *out = nullptr;
        return EA_ERR_CUDA;
    }
    return EA_OK;
}

int ea_set_schedule(ea_ctx *c, const uint64_t *t_w, int n_tw, const uint64_t *t, int n_t)
{
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (c->quenched)
        return fail(c, EA_ERR_STATE, "ea_set_schedule after ea_quench");
    if (n_tw < 0 || n_t < 0 || n_tw > ea::kMaxSchedule || n_t > ea::kMaxSchedule ||
        (n_tw > 0 && !t_w) || (n_t > 0 && !t))
        return fail(c, EA_ERR_INVALID_ARG, "bad schedule arrays");
    for (int i = 0; i < n_tw; ++i)
        if (t_w[i] >= ea::kMaxTime)
            return fail(c, EA_ERR_INVALID_ARG, "waiting time >= 2^48");
    for (int i = 0; i < n_t; ++i)
        if (t[i] >= ea::kMaxTime)
            return fail(c, EA_ERR_INVALID_ARG, "time lag >= 2^48");
    return build_schedule(c, sorted_unique(t_w, n_tw), sorted_unique(t, n_t));
}

int ea_quench(ea_ctx *c, double T, int rule)
{
    NvtxRange nvtx_range("ea_quench");
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    uint64_t thr[7];
    uint8_t alw[7];
    if (compute_thresholds(T, rule, thr, alw) != EA_OK)
        return fail(c, EA_ERR_INVALID_ARG, "bad temperature or rule");
    c->T = T;
    c->rule = rule;
    std::memcpy(c->thr_k, thr, sizeof(thr));
    std::memcpy(c->always_k, alw, sizeof(alw));
    c->thr = make_thr(rule, T, thr, alw);
    ea::fill_job_thresholds(&c->jd, c->thr);
    EA_CUDA(c, ea::launch_init_spins(c->spins, c->geo, c->first, c->S, c->seed, c->stream));
    if (c->res)
        EA_CUDA(c, cudaMemsetAsync(c->res, 0, c->res_bytes, c->stream));
    ++c->res_gen;
    c->t = 0;
    c->quenched = true;
    int rc = upload_job(c);
    if (rc != EA_OK)
        return rc;
    return fire_measurements(c, c->stream);
}

int ea_sweep(ea_ctx *c, uint64_t n)
{
    NvtxRange nvtx_range("ea_sweep");
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_sweep before ea_quench");
    if (n > ea::kMaxTime || c->t + n > ea::kMaxTime)
        return fail(c, EA_ERR_INVALID_ARG, "time would pass 2^48");
    if (c->half != 0)
        return fail(c, EA_ERR_STATE, "ea_sweep between the half-steps of ea_half_sweep");
    const uint64_t target = c->t + n;
    while (c->t < target) {
        auto it = std::upper_bound(c->meas.begin(), c->meas.end(), c->t);
        const uint64_t stop = (it == c->meas.end()) ? target : std::min(target, *it);
        int rc0 = upload_time(c, stop);
        if (rc0 != EA_OK)
            return rc0;
        rc0 = launch_plain(c, stop - c->t);
        if (rc0 != EA_OK)
            return rc0;
        c->t = stop;
        const int rc = fire_measurements(c, c->stream);
        if (rc != EA_OK)
            return rc;
    }
    return EA_OK;
}

int ea_set_row_range(ea_ctx *c, int y_lo, int y_hi)
{
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (c->L != 64 && c->L != 128)
        return fail(c, EA_ERR_INVALID_ARG, "ea_set_row_range: sides 64 and 128 only");
    if (y_lo < 0 || y_hi > c->geo.n[1] || y_lo >= y_hi)
        return fail(c, EA_ERR_INVALID_ARG, "ea_set_row_range: need 0 <= y_lo < y_hi <= L");
    if (!c->tw.empty() || !c->tt.empty())
        return fail(c, EA_ERR_STATE, "ea_set_row_range on a context with a measurement schedule");
    if (c->batch)
        return fail(c, EA_ERR_STATE, "ea_set_row_range on a member of a batch");
    c->jd.row_lo = y_lo;
    c->jd.row_hi = y_hi;
    return EA_OK;
}

int ea_half_sweep(ea_ctx *c)
{
    NvtxRange nvtx_range("ea_half_sweep");
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_half_sweep before ea_quench");
    if (!c->meas.empty())
        return fail(c, EA_ERR_STATE, "ea_half_sweep on a context with a measurement schedule");
    if (c->batch)
        return fail(c, EA_ERR_STATE, "ea_half_sweep on a member of a batch");
    if (c->t + 1 > ea::kMaxTime)
        return fail(c, EA_ERR_INVALID_ARG, "time would pass 2^48");
    if (c->half == 0) {
        const int rc = upload_time(c, c->t + 1);
        if (rc != EA_OK)
            return rc;
    }
    const bool heat = c->rule == EA_RULE_HEATBATH;
    EA_CUDA(c, ea::launch_sweep_table(heat ? nullptr : &c->jd, heat ? nullptr : c->jd_dev,
                                      heat ? 0 : 1, heat ? &c->jd : nullptr,
                                      heat ? c->jd_dev : nullptr, heat ? 1 : 0, 1, c->stream,
                                      nullptr, nullptr, c->half));
    if (c->half == 1) {
        c->half = 0;
        c->t += 1;
    } else {
        c->half = 1;
    }
    return EA_OK;
}

// Rows y .. y + n_rows - 1 of one area of every sample, host layout
// [sample][z'][row][x'] (word-lattice words).
static int copy_rows(ea_ctx *c, int area, int y, int n_rows, uint32_t *host, bool to_host)
{
    if (check_ctx(c) || !host || (area != 0 && area != 1) || n_rows < 1 || y < 0 ||
        y + n_rows > c->geo.n[1])
        return EA_ERR_INVALID_ARG;
    const size_t n0 = (size_t)c->geo.n[0], n2 = (size_t)c->geo.n[2];
    const size_t sz = n0 * (size_t)c->geo.n[1], W = (size_t)c->geo.words;
    const size_t width = (size_t)n_rows * n0 * sizeof(uint32_t);
    for (int s = 0; s < c->S; ++s) {
        uint32_t *dev = c->spins + ((size_t)s * 2 + area) * W + (size_t)y * n0;
        uint32_t *h = host + (size_t)s * n2 * n_rows * n0;
        const cudaError_t e =
            to_host ? cudaMemcpy2DAsync(h, width, dev, sz * sizeof(uint32_t), width, n2,
                                        cudaMemcpyDeviceToHost, c->stream)
                    : cudaMemcpy2DAsync(dev, sz * sizeof(uint32_t), h, width, width, n2,
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, to_host ? "ea_get_rows" : "ea_set_rows");
    }
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!to_host)
        ++c->res_gen;
    return EA_OK;
}

int ea_get_rows(ea_ctx *c, int area, int y, int n_rows, uint32_t *host_words)
{
    return copy_rows(c, area, y, n_rows, host_words, true);
}

int ea_set_rows(ea_ctx *c, int area, int y, int n_rows, const uint32_t *host_words)
{
    return copy_rows(c, area, y, n_rows, const_cast<uint32_t *>(host_words), false);
}

int ea_time(const ea_ctx *c, uint64_t *t)
{
    if (!c || !t)
        return EA_ERR_INVALID_ARG;
    *t = c->t;
    return EA_OK;
}

int ea_measure(ea_ctx *c, uint64_t t_w, uint64_t t, ea_obs *out)
{
    NvtxRange nvtx_range("ea_measure");
    if (check_ctx(c) || !out)
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_measure before ea_quench");
    const int i = idx_of(c->tw, t_w), j = idx_of(c->tt, t);
    if (i < 0 || j < 0 || t_w + t > c->t)
        return fail(c, EA_ERR_NO_SNAPSHOT, "(t_w, t) not scheduled or not reached");
    const int mi = idx_of(c->meas, t_w + t);
    const size_t S = (size_t)c->S, R = (size_t)c->R();
    const long long N = (long long)c->L * c->L * c->L;
    // all of the job's sums in one copy, reused until new sums are made
    if (c->res_host_gen != c->res_gen) {
        c->res_host.resize(c->res_bytes / sizeof(unsigned long long));
        EA_CUDA(c, cudaMemcpyAsync(c->res_host.data(), c->res, c->res_bytes,
                                   cudaMemcpyDeviceToHost, c->stream));
        EA_CUDA(c, cudaStreamSynchronize(c->stream));
        c->res_host_gen = c->res_gen;
    }
    const unsigned long long *res = c->res_host.data();
    const size_t slot_a = c->off_a + ((size_t)i * c->tt.size() + (size_t)j) * S * 2;
    const std::vector<unsigned long long> a(res + slot_a, res + slot_a + S * 2);
    const std::vector<unsigned long long> q(res + c->off_q + mi * S, res + c->off_q + mi * S + S);
    const std::vector<unsigned long long> u(res + c->off_u + mi * S * 2,
                                            res + c->off_u + mi * S * 2 + S * 2);
    const std::vector<unsigned long long> gp(res + c->off_g + (size_t)i * S * 3 * R,
                                             res + c->off_g + (size_t)(i + 1) * S * 3 * R);

    // integer observables: N - 2 * (number of differing sites), and
    // H = (unsatisfied bonds) - (satisfied bonds) = 2 U - 3N
    double Csum = 0.0, qsum = 0.0;
    long long Atot = 0;
    for (size_t k = 0; k < S * 2; ++k) {
        const long long A = N - 2 * (long long)a[k];
        Atot += A;
        if (out->A)
            out->A[k] = A;
        if (out->E)
            out->E[k] = 2 * (long long)u[k] - 3 * N;
    }
    for (size_t s = 0; s < S; ++s) {
        const long long Q = N - 2 * (long long)q[s];
        if (out->Q)
            out->Q[s] = Q;
        qsum += (double)Q / (double)N;
    }
    Csum = (double)Atot / (double)(N * 2 * (long long)S);
    out->C = Csum;
    out->q_mean = qsum / (double)S;

    // C4 (Eq. 3): average over axes and samples; SEM over samples
    std::vector<long long> G(S * 3 * R);
    for (size_t k = 0; k < G.size(); ++k)
        G[k] = N - 2 * (long long)gp[k];
    if (out->G)
        for (size_t k = 0; k < G.size(); ++k)
            out->G[k] = G[k];
    std::vector<double> c4(R), sem(R);
    for (size_t r = 0; r < R; ++r) {
        long long tot = 0;
        for (size_t s = 0; s < S; ++s)
            for (int d = 0; d < 3; ++d)
                tot += G[(s * 3 + d) * R + r];
        c4[r] = (double)tot / (3.0 * (double)N * (double)S);
        if (S >= 2) {
            std::vector<double> ps(S);
            double mean = 0.0;
            for (size_t s = 0; s < S; ++s) {
                long long v = 0;
                for (int d = 0; d < 3; ++d)
                    v += G[(s * 3 + d) * R + r];
                ps[s] = (double)v / (3.0 * (double)N);
                mean += ps[s];
            }
            mean /= (double)S;
            double ss = 0.0;
            for (size_t s = 0; s < S; ++s)
                ss += (ps[s] - mean) * (ps[s] - mean);
            sem[r] = std::sqrt(ss / (double)(S - 1)) / std::sqrt((double)S);
        } else {
            sem[r] = NAN;
        }
    }
    // cut where C4 first drops below three times its error (Sec. IV)
    int rc = (int)R - 1;
    if (S >= 2) {
        for (int r = 1; r < (int)R; ++r)
            if (c4[r] < 3.0 * sem[r]) {
                rc = r - 1;
                break;
            }
    }
    double I1 = 0.0, I2 = 0.0;
    for (int r = 1; r <= rc; ++r) {
        I1 += r * c4[r];
        I2 += (double)r * r * c4[r];
    }
    out->r_cut = rc;
    out->xi1 = (rc < 1 || I1 == 0.0) ? NAN : I2 / I1;
    if (out->C4)
        for (size_t r = 0; r < R; ++r)
            out->C4[r] = c4[r];
    if (out->C4_sem)
        for (size_t r = 0; r < R; ++r)
            out->C4_sem[r] = sem[r];
    return EA_OK;
}

int ea_c4_radial_bins(int L, int *n_bins)
{
    if (!n_bins || L < 2 || (L & 1) || L > ea::kC4FullMaxL)
        return EA_ERR_INVALID_ARG;
    *n_bins = 3 * (L / 2) * (L / 2) + 1;
    return EA_OK;
}

// Vectors per squared distance r^2 of side L: a shortest-image component m
// stands for d = m and d = L - m, one vector when they coincide (m = 0 or L/2).
static void c4_radial_counts(int L, long long *counts)
{
    const int H = L / 2, n_bins = 3 * H * H + 1;
    std::fill(counts, counts + n_bins, 0LL);
    auto images = [H](int m) { return (m == 0 || m == H) ? 1LL : 2LL; };
    for (int mz = 0; mz <= H; ++mz)
        for (int my = 0; my <= H; ++my)
            for (int mx = 0; mx <= H; ++mx)
                counts[mx * mx + my * my + mz * mz] += images(mx) * images(my) * images(mz);
}

// The FP64 curve of the all-vector sums (Eq. 3 over every displacement vector
// of length r): for a bin with vectors, C4 = sum_s sums[s][b] / (counts[b] N S)
// and sem the standard error over samples of sums[s][b] / (counts[b] N) (NaN
// for one sample); a bin with no vector gets NaN in both.  Either output may
// be NULL.
static void c4_radial_curve(const long long *sums, const long long *counts, int S, int n_bins,
                            double N, double *C4, double *sem)
{
    if (!C4 && !sem)
        return;
    std::vector<double> ps((size_t)S);
    for (int b = 0; b < n_bins; ++b) {
        if (counts[b] == 0) {
            if (C4)
                C4[b] = NAN;
            if (sem)
                sem[b] = NAN;
            continue;
        }
        const double norm = (double)counts[b] * N;
        long long tot = 0;
        for (int s = 0; s < S; ++s)
            tot += sums[(size_t)s * n_bins + b];
        if (C4)
            C4[b] = (double)tot / (norm * (double)S);
        if (!sem)
            continue;
        if (S < 2) {
            sem[b] = NAN;
            continue;
        }
        double mean = 0.0;
        for (int s = 0; s < S; ++s) {
            ps[s] = (double)sums[(size_t)s * n_bins + b] / norm;
            mean += ps[s];
        }
        mean /= (double)S;
        double ss = 0.0;
        for (int s = 0; s < S; ++s)
            ss += (ps[s] - mean) * (ps[s] - mean);
        sem[b] = std::sqrt(ss / (double)(S - 1)) / std::sqrt((double)S);
    }
}

int ea_c4_radial(ea_ctx *c, uint64_t t_w, long long *sums, long long *counts, double *C4,
                 double *C4_sem)
{
    NvtxRange nvtx_range("ea_c4_radial");
    if (check_ctx(c) || !sums || !counts)
        return EA_ERR_INVALID_ARG;
    if (c->L > ea::kC4FullMaxL)
        return fail(c, EA_ERR_INVALID_ARG, "ea_c4_radial: side above 512");
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_c4_radial before ea_quench");
    const int i = idx_of(c->tw, t_w);
    if (i < 0 || t_w > c->t)
        return fail(c, EA_ERR_NO_SNAPSHOT, "t_w not scheduled or not reached");
    const int L = c->L, H = L / 2, n_bins = 3 * H * H + 1;
    c4_radial_counts(L, counts);
    ea::C4FullTables fwd, inv;
    if (ea::make_c4full_plan(L, &fwd, &inv) != 0)
        return fail(c, EA_ERR_INVALID_ARG, "ea_c4_radial: no transform prime for this side");
    const size_t per = ea::c4full_scratch_words(L);
    const int chunk = (int)std::max<size_t>(
        1, std::min<size_t>((size_t)c->S, ((size_t)256 << 20) / (per * sizeof(uint32_t))));
    const size_t scratch_bytes = (size_t)chunk * per * sizeof(uint32_t);
    const size_t bins_bytes = (size_t)c->S * n_bins * sizeof(long long);
    uint32_t *scratch = (uint32_t *)dev_alloc(scratch_bytes, c->stream);
    long long *bins = (long long *)dev_alloc(bins_bytes, c->stream);
    auto release = [&]() {
        dev_free(scratch, scratch_bytes, c->stream);
        dev_free(bins, bins_bytes, c->stream);
    };
    if (!scratch || !bins) {
        release();
        return fail(c, EA_ERR_OOM, "ea_c4_radial: scratch allocation failed");
    }
    cudaError_t err = cudaMemsetAsync(bins, 0, bins_bytes, c->stream);
    const uint32_t *snap = c->snaps + (size_t)i * c->area_words();
    for (int s0 = 0; s0 < c->S && err == cudaSuccess; s0 += chunk)
        err = ea::launch_c4full(snap, c->geo, s0, std::min(chunk, c->S - s0), scratch, fwd, inv,
                                bins, n_bins, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(sums, bins, bins_bytes, cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(c->stream);
    release();
    if (err != cudaSuccess)
        return cuda_fail(c, err, "ea_c4_radial");
    c4_radial_curve(sums, counts, c->S, n_bins, (double)L * L * L, C4, C4_sem);
    return EA_OK;
}

int ea_c4_radial_noalloc(ea_ctx *c, uint64_t t_w, long long *sums, long long *counts, double *C4,
                         double *C4_sem)
{
    NvtxRange nvtx_range("ea_c4_radial_noalloc");
    if (check_ctx(c) || !sums || !counts)
        return EA_ERR_INVALID_ARG;
    if (c->L > ea::kC4FullNoAllocMaxL)
        return fail(c, EA_ERR_INVALID_ARG,
                    "ea_c4_radial_noalloc: side above 128, the size of its static scratch");
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_c4_radial_noalloc before ea_quench");
    const int i = idx_of(c->tw, t_w);
    if (i < 0 || t_w > c->t)
        return fail(c, EA_ERR_NO_SNAPSHOT, "t_w not scheduled or not reached");
    const int L = c->L, H = L / 2, n_bins = 3 * H * H + 1;
    c4_radial_counts(L, counts);
    ea::C4FullTables fwd, inv;
    if (ea::make_c4full_plan(L, &fwd, &inv) != 0)
        return fail(c, EA_ERR_INVALID_ARG,
                    "ea_c4_radial_noalloc: no transform prime for this side");
    long long *bins = nullptr;
    uint32_t *residues = nullptr;
    cudaError_t err = ea::c4full_static_scratch(&bins, &residues);
    if (err != cudaSuccess)
        return cuda_fail(c, err, "ea_c4_radial_noalloc: static scratch address");
    // one sample at a time through the shared scratch, in stream order; the
    // bins left by the previous sample or call are cleared first
    const size_t W = (size_t)c->geo.words;
    const uint32_t *snap = c->snaps + (size_t)i * c->area_words();
    const size_t row_bytes = (size_t)n_bins * sizeof(long long);
    for (int s = 0; s < c->S && err == cudaSuccess; ++s) {
        err = cudaMemsetAsync(bins, 0, row_bytes, c->stream);
        if (err == cudaSuccess)
            err = ea::launch_c4full(snap + (size_t)s * 2 * W, c->geo, 0, 1, residues, fwd, inv,
                                    bins, n_bins, c->stream);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(sums + (size_t)s * n_bins, bins, row_bytes,
                                  cudaMemcpyDeviceToHost, c->stream);
    }
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess)
        return cuda_fail(c, err, "ea_c4_radial_noalloc");
    c4_radial_curve(sums, counts, c->S, n_bins, (double)L * L * L, C4, C4_sem);
    return EA_OK;
}

int ea_get_spins(ea_ctx *c, int s, int a, int8_t *out)
{
    if (check_ctx(c) || !out || s < 0 || s >= c->S || a < 0 || a > 1)
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_get_spins before ea_quench");
    const Geo &g = c->geo;
    const size_t W = (size_t)g.words;
    std::vector<uint32_t> h(2 * W);
    EA_CUDA(c, cudaMemcpyAsync(h.data(), c->spins + (size_t)s * 2 * W, 2 * W * 4,
                               cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    const int L = c->L;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int xw = x % g.n[0], yw = y % g.n[1], zw = z % g.n[2];
                const int b = x / g.n[0] + g.k[0] * (y / g.n[1] + g.k[1] * (z / g.n[2]));
                const size_t w = (size_t)xw + (size_t)g.n[0] * (yw + (size_t)g.n[1] * zw);
                const int col = (xw + yw + zw) & 1;
                const uint32_t bit = (h[(size_t)(a ^ col) * W + w] >> b) & 1u;
                out[(size_t)x + (size_t)L * (y + (size_t)L * z)] = bit ? -1 : 1;
            }
    return EA_OK;
}

int ea_get_couplings(ea_ctx *c, int s, int8_t *out)
{
    if (check_ctx(c) || !out || s < 0 || s >= c->S)
        return EA_ERR_INVALID_ARG;
    const Geo &g = c->geo;
    const size_t W = (size_t)g.words;
    std::vector<uint32_t> h(3 * W);
    EA_CUDA(c, cudaMemcpyAsync(h.data(), c->J + (size_t)s * 3 * W, 3 * W * 4,
                               cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    const int L = c->L;
    const size_t N = (size_t)L * L * L;
    for (int d = 0; d < 3; ++d)
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int xw = x % g.n[0], yw = y % g.n[1], zw = z % g.n[2];
                    const int b = x / g.n[0] + g.k[0] * (y / g.n[1] + g.k[1] * (z / g.n[2]));
                    const size_t w = (size_t)xw + (size_t)g.n[0] * (yw + (size_t)g.n[1] * zw);
                    const uint32_t bit = (h[(size_t)d * W + w] >> b) & 1u;
                    out[d * N + (size_t)x + (size_t)L * (y + (size_t)L * z)] = bit ? -1 : 1;
                }
    return EA_OK;
}

int ea_set_spins(ea_ctx *c, int s, int a, const int8_t *in)
{
    if (check_ctx(c) || !in || s < 0 || s >= c->S || a < 0 || a > 1)
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_set_spins before ea_quench");
    const Geo &g = c->geo;
    const size_t W = (size_t)g.words;
    std::vector<uint32_t> h(2 * W);
    EA_CUDA(c, cudaMemcpyAsync(h.data(), c->spins + (size_t)s * 2 * W, 2 * W * 4,
                               cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    const int L = c->L;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int8_t v = in[(size_t)x + (size_t)L * (y + (size_t)L * z)];
                if (v != 1 && v != -1)
                    return fail(c, EA_ERR_INVALID_ARG, "spin value other than +-1");
                const int xw = x % g.n[0], yw = y % g.n[1], zw = z % g.n[2];
                const int b = x / g.n[0] + g.k[0] * (y / g.n[1] + g.k[1] * (z / g.n[2]));
                const size_t w = (size_t)xw + (size_t)g.n[0] * (yw + (size_t)g.n[1] * zw);
                const int col = (xw + yw + zw) & 1;
                uint32_t &word = h[(size_t)(a ^ col) * W + w];
                word = (word & ~(1u << b)) | ((uint32_t)(v == -1) << b);
            }
    EA_CUDA(c, cudaMemcpyAsync(c->spins + (size_t)s * 2 * W, h.data(), 2 * W * 4,
                               cudaMemcpyHostToDevice, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    return EA_OK;
}

int ea_set_couplings(ea_ctx *c, int s, const int8_t *in)
{
    if (check_ctx(c) || !in || s < 0 || s >= c->S)
        return EA_ERR_INVALID_ARG;
    const Geo &g = c->geo;
    const size_t W = (size_t)g.words;
    const int L = c->L;
    const size_t N = (size_t)L * L * L;
    std::vector<uint32_t> h(3 * W, 0u);
    for (int d = 0; d < 3; ++d)
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int8_t v = in[d * N + (size_t)x + (size_t)L * (y + (size_t)L * z)];
                    if (v != 1 && v != -1)
                        return fail(c, EA_ERR_INVALID_ARG, "coupling value other than +-1");
                    const int xw = x % g.n[0], yw = y % g.n[1], zw = z % g.n[2];
                    const int b = x / g.n[0] + g.k[0] * (y / g.n[1] + g.k[1] * (z / g.n[2]));
                    const size_t w = (size_t)xw + (size_t)g.n[0] * (yw + (size_t)g.n[1] * zw);
                    h[(size_t)d * W + w] |= (uint32_t)(v == -1) << b;
                }
    EA_CUDA(c, cudaMemcpyAsync(c->J + (size_t)s * 3 * W, h.data(), 3 * W * 4,
                               cudaMemcpyHostToDevice, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    return EA_OK;
}

int ea_coupling_words(const ea_ctx *c, size_t *n_words)
{
    if (!c || !n_words)
        return EA_ERR_INVALID_ARG;
    *n_words = (size_t)c->S * 3 * c->geo.words;
    return EA_OK;
}

int ea_get_coupling_words(ea_ctx *c, uint32_t *host_words)
{
    if (check_ctx(c) || !host_words)
        return EA_ERR_INVALID_ARG;
    EA_CUDA(c, cudaMemcpyAsync(host_words, c->J, c->J_bytes, cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    return EA_OK;
}

int ea_set_coupling_words(ea_ctx *c, const uint32_t *host_words)
{
    if (check_ctx(c) || !host_words)
        return EA_ERR_INVALID_ARG;
    const uint32_t valid = c->geo.valid;
    if (valid != 0xffffffffu) {  // lanes past the word's sites must stay 0
        const size_t n = (size_t)c->S * 3 * c->geo.words;
        for (size_t i = 0; i < n; ++i)
            if (host_words[i] & ~valid)
                return fail(c, EA_ERR_INVALID_ARG, "coupling word with bits outside its lanes");
    }
    EA_CUDA(c, cudaMemcpyAsync(c->J, host_words, c->J_bytes, cudaMemcpyHostToDevice, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));
    return EA_OK;
}

int ea_set_time(ea_ctx *c, uint64_t t)
{
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_set_time before ea_quench");
    if (t >= ea::kMaxTime)
        return fail(c, EA_ERR_INVALID_ARG, "time >= 2^48");
    c->t = t;
    return EA_OK;
}

int ea_get_thresholds(const ea_ctx *c, uint64_t thr[7], uint8_t always[7])
{
    if (!c || !thr || !always)
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return EA_ERR_STATE;
    std::memcpy(thr, c->thr_k, sizeof(c->thr_k));
    std::memcpy(always, c->always_k, sizeof(c->always_k));
    return EA_OK;
}

// ---- checkpoint -----------------------------------------------------------
namespace {
constexpr char kMagic[8] = {'E', 'A', 'G', 'B', '3', '0', '0', '\2'};

struct CkptHeader {
    char magic[8];
    int32_t L, S, G, rule, first, pad;
    double p_neg, T;
    uint64_t seed, t;
    uint64_t n_tw, n_t;
    uint64_t spins_bytes, J_bytes, snaps_bytes, res_bytes;
};

bool write_dev(FILE *f, const void *dev, size_t bytes, cudaStream_t s, std::string &err)
{
    if (!bytes)
        return true;
    std::vector<char> h(bytes);
    if (cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = cudaGetErrorString(cudaGetLastError());
        return false;
    }
    return fwrite(h.data(), 1, bytes, f) == bytes;
}

bool read_dev(FILE *f, void *dev, size_t bytes, cudaStream_t s)
{
    if (!bytes)
        return true;
    std::vector<char> h(bytes);
    if (fread(h.data(), 1, bytes, f) != bytes)
        return false;
    if (cudaMemcpyAsync(dev, h.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}
}  // namespace

int ea_checkpoint(ea_ctx *c, const char *path)
{
    NvtxRange nvtx_range("ea_checkpoint");
    if (check_ctx(c) || !path)
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_checkpoint before ea_quench");
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.L = c->L;
    h.S = c->S;
    h.G = c->G;
    h.first = c->first;
    h.rule = c->rule;
    h.p_neg = c->p_neg;
    h.T = c->T;
    h.seed = c->seed;
    h.t = c->t;
    h.n_tw = c->tw.size();
    h.n_t = c->tt.size();
    h.spins_bytes = c->spins_bytes;
    h.J_bytes = c->J_bytes;
    h.snaps_bytes = c->snaps_bytes;
    h.res_bytes = c->res_bytes;
    FILE *f = fopen(path, "wb");
    if (!f)
        return fail(c, EA_ERR_IO, std::string("cannot open ") + path);
    std::string err;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
    ok = ok && fwrite(c->tw.data(), 8, c->tw.size(), f) == c->tw.size();
    ok = ok && fwrite(c->tt.data(), 8, c->tt.size(), f) == c->tt.size();
    ok = ok && write_dev(f, c->spins, c->spins_bytes, c->stream, err);
    ok = ok && write_dev(f, c->J, c->J_bytes, c->stream, err);
    ok = ok && write_dev(f, c->snaps, c->snaps_bytes, c->stream, err);
    ok = ok && write_dev(f, c->res, c->res_bytes, c->stream, err);
    ok = (fclose(f) == 0) && ok;
    if (!ok)
        return fail(c, EA_ERR_IO, "checkpoint write failed " + err);
    return EA_OK;
}

int ea_restore(ea_ctx **out, const char *path, void *cuda_stream)
{
    if (!out || !path)
        return EA_ERR_INVALID_ARG;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f)
        return EA_ERR_IO;
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 ||
        h.n_tw > (uint64_t)ea::kMaxSchedule || h.n_t > (uint64_t)ea::kMaxSchedule) {
        fclose(f);
        return EA_ERR_IO;
    }
    std::vector<uint64_t> tw(h.n_tw), tt(h.n_t);
    if (fread(tw.data(), 8, h.n_tw, f) != h.n_tw || fread(tt.data(), 8, h.n_t, f) != h.n_t) {
        fclose(f);
        return EA_ERR_IO;
    }
    ea_ctx *c = nullptr;
    int rc = ea_create_samples_range(&c, h.L, h.p_neg, h.seed, h.first, h.S, h.G, cuda_stream);
    if (rc != EA_OK) {
        fclose(f);
        return rc;
    }
    rc = ea_set_schedule(c, tw.data(), (int)tw.size(), tt.data(), (int)tt.size());
    if (rc == EA_OK && (h.spins_bytes != c->spins_bytes || h.J_bytes != c->J_bytes ||
                        h.snaps_bytes != c->snaps_bytes || h.res_bytes != c->res_bytes))
        rc = EA_ERR_IO;
    if (rc == EA_OK) {
        uint64_t thr[7];
        uint8_t alw[7];
        if (compute_thresholds(h.T, h.rule, thr, alw) != EA_OK)
            rc = EA_ERR_IO;
        else {
            c->T = h.T;
            c->rule = h.rule;
            std::memcpy(c->thr_k, thr, sizeof(thr));
            std::memcpy(c->always_k, alw, sizeof(alw));
            c->thr = make_thr(h.rule, h.T, thr, alw);
            ea::fill_job_thresholds(&c->jd, c->thr);
        }
    }
    if (rc == EA_OK) {
        bool ok = read_dev(f, c->spins, c->spins_bytes, c->stream) &&
                  read_dev(f, c->J, c->J_bytes, c->stream) &&
                  read_dev(f, c->snaps, c->snaps_bytes, c->stream) &&
                  read_dev(f, c->res, c->res_bytes, c->stream);
        ++c->res_gen;
        if (!ok)
            rc = EA_ERR_IO;
    }
    fclose(f);
    if (rc != EA_OK) {
        ea_destroy(c);
        return rc;
    }
    c->t = h.t;
    c->quenched = true;
    rc = upload_job(c);
    if (rc != EA_OK) {
        ea_destroy(c);
        return rc;
    }
    *out = c;
    return EA_OK;
}

int ea_destroy(ea_ctx *c)
{
    if (!c)
        return EA_OK;
    if (c->batch)
        ea_batch_remove(c->batch, c);
    if (c->spins || c->J || c->snaps || c->res || c->jd_dev)
        cudaStreamSynchronize(c->stream);
    release_schedule(c);
    dev_free(c->spins, c->spins_bytes, c->stream);
    dev_free(c->J, c->J_bytes, c->stream);
    dev_free(c->jd_dev, sizeof(ea::JobDev), c->stream);
    delete c;
    return EA_OK;
}

const char *ea_last_error(const ea_ctx *c)
{
    if (!c)
        return "";
    return c->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct ea_batch {
    cudaStream_t stream = nullptr;
    std::vector<ea_ctx *> members;
    int cpt = 0;           // word columns per thread (0 = per-job default)
    int graph_sweeps = 0;  // sweeps per captured graph (0 = direct launches)
    int res_max_L = ea::kResDefaultMaxL;  // Metropolis sides up to this run sample-resident
    int variant = 0;                      // bit 0: side 128 on the staged kernel
    // a table of one kernel's jobs is split over this many streams (1 .. 5)
    int streams = ea::kDefaultStreams;
    // device job tables, one per update rule
    ea::JobDev *tab_dev[2] = {nullptr, nullptr};
    size_t cap[2] = {0, 0};
    int n_jobs[2] = {0, 0};
    std::vector<ea::JobDev> tab_host[2];
    uint64_t tab_sig = 0;  // what the launches take from the host tables (table_signature)
    // captured graph of graph_sweeps sweeps over the current tables
    cudaGraphExec_t graph = nullptr;
    int graph_K = 0;
    uint64_t graph_kernels = 0;  // kernels per replay
    const void *graph_key[2] = {nullptr, nullptr};
    uint64_t graph_sig = 0;
    int graph_streams = 0;
    // side streams: the runs of a mixed table (column kernel, general tiles,
    // side 64, side 128) are enqueued concurrently
    ea::SideStreams side{};
    bool have_side = false;
    std::string err;
};

namespace {

int bfail(ea_batch *b, int code, const std::string &msg)
{
    if (b)
        b->err = msg;
    return code;
}

#define EA_BCUDA(b, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cudaGetLastError();                                                        \
            return bfail((b), EA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                              \
    } while (0)

void drop_graph(ea_batch *b)
{
    if (b->graph)
        cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_K = 0;
}

// A hash of everything a captured graph's launches take from the host tables
// at capture time (order, pointers, keys, geometry, launch shape, class flags
// and the kernel variant chosen from the tables), not the times, which the
// launches read from the device rows.  A graph is replayed only while it
// matches.
uint64_t table_signature(const std::vector<ea::JobDev> (&tab)[2])
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a, 64 bit
    auto mix = [&h](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xFFu;
            h *= 1099511628211ull;
        }
    };
    for (int r = 0; r < 2; ++r) {
        mix(0xA5A5u + (uint64_t)r);
        mix(tab[r].size());
        for (const ea::JobDev &jd : tab[r]) {
            mix((uint64_t)(uintptr_t)jd.spins);
            mix((uint64_t)(uintptr_t)jd.J);
            mix(((uint64_t)jd.rk[0] << 32) | jd.rk[1]);
            mix(((uint64_t)(uint32_t)jd.geo.L << 32) | (uint32_t)jd.n_samples);
            mix(((uint64_t)jd.rng_group << 32) | (uint32_t)jd.cols_per_thread);
            mix(((uint64_t)jd.geo_live << 32) | jd.always_u);
            mix(((uint64_t)(uint32_t)jd.all_always << 32) | (uint32_t)jd.none_random);
            mix(((uint64_t)jd.gC_hi[1][32] << 32) | jd.gC_hi[0][32]);
            mix(((uint64_t)(uint32_t)jd.resident << 32) | (uint32_t)jd.variant);
            mix(((uint64_t)(uint32_t)jd.row_lo << 32) | (uint32_t)jd.row_hi);
        }
    }
    return h;
}

// Rebuild both rule tables from the members' current state and upload them;
// member i may run up to min(n, limits[i]) more sweeps (limits may be NULL).
int upload_tables(ea_batch *b, uint64_t n, const std::vector<uint64_t> *limits = nullptr)
{
    size_t mi = 0;
    for (int r = 0; r < 2; ++r)
        b->tab_host[r].clear();
    for (ea_ctx *m : b->members) {
        const int r = m->rule == EA_RULE_HEATBATH ? 1 : 0;
        ea::JobDev jd = m->jd;
        jd.t = m->t;
        uint64_t allow = std::min<uint64_t>(n, ea::kMaxTime - m->t);
        if (limits)
            allow = std::min<uint64_t>(allow, (*limits)[mi]);
        ++mi;
        jd.t_end = m->t + allow;
        if (b->cpt > 0)
            ea::fill_job_layout(&jd, b->cpt);
        jd.resident = (r == 0 && jd.geo.L <= b->res_max_L && ea::res_side_fits(jd.geo.L) &&
                       jd.row_lo == 0 && jd.row_hi == jd.geo.n[1])
                          ? 1
                          : 0;
        jd.variant = b->variant;
        b->tab_host[r].push_back(jd);
    }
    // equal sides next to each other: the sample-resident jobs first, then the
    // sides of the column kernels, those of the general tile kernel next, sides
    // 64 and 128 last (their own tile kernels); the order of rows changes no
    // result
    auto run_key = [](const ea::JobDev &jd) {
        const int L = jd.geo.L;
        if (jd.resident)
            return L;
        return (L == 64 || L == 128) ? (3 << 20) + L
               : ea::general_tile_side(L) ? (2 << 20) + L
                                          : (1 << 20) + L;
    };
    for (int r = 0; r < 2; ++r)
        std::stable_sort(b->tab_host[r].begin(), b->tab_host[r].end(),
                         [&](const ea::JobDev &a, const ea::JobDev &c) {
                             return run_key(a) < run_key(c);
                         });
    b->tab_sig = table_signature(b->tab_host);
    for (int r = 0; r < 2; ++r) {
        const size_t n = b->tab_host[r].size();
        b->n_jobs[r] = (int)n;
        if (n == 0)
            continue;
        if (n > b->cap[r]) {
            size_t cap = std::max<size_t>(n, 2 * b->cap[r]);
            dev_free(b->tab_dev[r], b->cap[r] * sizeof(ea::JobDev), b->stream);
            b->tab_dev[r] = (ea::JobDev *)dev_alloc(cap * sizeof(ea::JobDev), b->stream);
            b->cap[r] = cap;
            if (!b->tab_dev[r])
                return bfail(b, EA_ERR_OOM, "batch table allocation failed");
        }
        EA_BCUDA(b, cudaMemcpyAsync(b->tab_dev[r], b->tab_host[r].data(), n * sizeof(ea::JobDev),
                                    cudaMemcpyHostToDevice, b->stream));
    }
    return EA_OK;
}

int enqueue_direct(ea_batch *b, uint64_t n, unsigned long long *counters = nullptr)
{
    EA_BCUDA(b, ea::launch_sweep_table(b->tab_host[0].data(), b->tab_dev[0], b->n_jobs[0],
                                       b->tab_host[1].data(), b->tab_dev[1], b->n_jobs[1], n,
                                       b->stream, counters, b->have_side ? &b->side : nullptr,
                                       -1, b->streams));
    for (int r = 0; r < 2; ++r)
        EA_BCUDA(b, ea::launch_advance_time(b->tab_dev[r], b->n_jobs[r], n, b->stream));
    return EA_OK;
}

int ensure_graph(ea_batch *b)
{
    const int K = b->graph_sweeps;
    if (b->graph && b->graph_K == K && b->graph_key[0] == b->tab_dev[0] &&
        b->graph_key[1] == b->tab_dev[1] && b->graph_sig == b->tab_sig &&
        b->graph_streams == b->streams)
        return EA_OK;
    drop_graph(b);
    cudaGraph_t g = nullptr;
    EA_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    ea::capture_begin();
    const int rc = enqueue_direct(b, (uint64_t)K);
    const uint64_t kernels = ea::capture_end();
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != EA_OK || e != cudaSuccess) {
        cudaGetLastError();
        if (g)
            cudaGraphDestroy(g);
        return bfail(b, EA_ERR_CUDA, "graph capture failed");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        return bfail(b, EA_ERR_CUDA, "graph instantiation failed");
    }
    b->graph_K = K;
    b->graph_kernels = kernels;
    b->graph_key[0] = b->tab_dev[0];
    b->graph_key[1] = b->tab_dev[1];
    b->graph_sig = b->tab_sig;
    b->graph_streams = b->streams;
    return EA_OK;
}

// n sweeps of every member on the tables as uploaded (no measurements).
int run_sweeps(ea_batch *b, uint64_t n)
{
    if (n == 0 || (b->n_jobs[0] == 0 && b->n_jobs[1] == 0))
        return EA_OK;
    uint64_t rem = n;
    if (b->graph_sweeps > 0 && b->stream != nullptr && n >= (uint64_t)b->graph_sweeps) {
        int rc = ensure_graph(b);
        if (rc != EA_OK)
            return rc;
        const uint64_t full = n / (uint64_t)b->graph_sweeps;
        for (uint64_t i = 0; i < full; ++i) {
            EA_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
            ea::count_launches(b->graph_kernels);
        }
        rem = n - full * (uint64_t)b->graph_sweeps;
    }
    if (rem)
        return enqueue_direct(b, rem);
    return EA_OK;
}

}  // namespace

extern "C" {

uint64_t ea_launch_count(void)
{
    return ea::launches_total();
}

int ea_batch_create(ea_batch **out, void *cuda_stream)
{
    if (!out)
        return EA_ERR_INVALID_ARG;
    ea_batch *b = new (std::nothrow) ea_batch();
    if (!b)
        return EA_ERR_OOM;
    b->stream = (cudaStream_t)cuda_stream;
    // without side streams a mixed table runs its parts one after another
    bool ok = true;
    for (int i = 0; i < ea::kSideStreams; ++i)
        ok = ok && cudaStreamCreateWithFlags(&b->side.stream[i], cudaStreamNonBlocking) ==
                       cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->side.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < ea::kSideStreams; ++i)
        ok = ok && cudaEventCreateWithFlags(&b->side.join[i], cudaEventDisableTiming) == cudaSuccess;
    cudaGetLastError();
    b->have_side = ok;
    *out = b;
    return EA_OK;
}

int ea_batch_add(ea_batch *b, ea_ctx *job)
{
    if (!b || !job || job->batch)
        return b ? bfail(b, EA_ERR_INVALID_ARG, "job is NULL or already in a batch")
                 : EA_ERR_INVALID_ARG;
    if (!job->quenched)
        return bfail(b, EA_ERR_STATE, "job not quenched");
    // work already queued on the job's own stream must come first
    if (job->stream != b->stream)
        EA_BCUDA(b, cudaStreamSynchronize(job->stream));
    job->batch = b;
    job->stream = b->stream;
    b->members.push_back(job);
    return EA_OK;
}

int ea_batch_remove(ea_batch *b, ea_ctx *job)
{
    if (!b || !job)
        return EA_ERR_INVALID_ARG;
    auto it = std::find(b->members.begin(), b->members.end(), job);
    if (it == b->members.end())
        return bfail(b, EA_ERR_INVALID_ARG, "job is not a member");
    if (job->own_stream != b->stream)
        EA_BCUDA(b, cudaStreamSynchronize(b->stream));
    b->members.erase(it);
    job->batch = nullptr;
    job->stream = job->own_stream;
    return EA_OK;
}

int ea_batch_size(const ea_batch *b, int *n_jobs)
{
    if (!b || !n_jobs)
        return EA_ERR_INVALID_ARG;
    *n_jobs = (int)b->members.size();
    return EA_OK;
}

int ea_batch_configure(ea_batch *b, int cols_per_thread, int graph_sweeps)
{
    if (!b || !(cols_per_thread == 0 || cols_per_thread == 1 || cols_per_thread == 2 ||
                cols_per_thread == 4) ||
        graph_sweeps < 0 || graph_sweeps > 4096)
        return EA_ERR_INVALID_ARG;
    b->cpt = cols_per_thread;
    b->graph_sweeps = graph_sweeps;
    return EA_OK;
}

int ea_batch_get_config(const ea_batch *b, int *cols_per_thread, int *graph_sweeps)
{
    if (!b || !cols_per_thread || !graph_sweeps)
        return EA_ERR_INVALID_ARG;
    *cols_per_thread = b->cpt;
    *graph_sweeps = b->graph_sweeps;
    return EA_OK;
}

}  // extern "C"

namespace {

// n sweeps of every member, member i stopping after limits[i] of them (all n
// when limits is NULL); scheduled measurements fire at each member's times.
int batch_sweep_impl(ea_batch *b, uint64_t n, const std::vector<uint64_t> *limits)
{
    for (size_t i = 0; i < b->members.size(); ++i) {
        ea_ctx *m = b->members[i];
        const uint64_t want = limits ? std::min<uint64_t>(n, (*limits)[i]) : n;
        if (want > ea::kMaxTime || m->t + want > ea::kMaxTime)
            return bfail(b, EA_ERR_INVALID_ARG, "a member's time would pass 2^48");
    }
    if (b->members.empty() || n == 0)
        return EA_OK;
    std::vector<uint64_t> end(b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i)
        end[i] = b->members[i]->t + (limits ? std::min<uint64_t>(n, (*limits)[i]) : n);
    int rc = upload_tables(b, n, limits);
    if (rc != EA_OK)
        return rc;
    uint64_t remaining = n;
    while (remaining > 0) {
        uint64_t step = remaining;
        bool any = false;
        for (size_t i = 0; i < b->members.size(); ++i) {
            ea_ctx *m = b->members[i];
            if (m->t >= end[i])
                continue;
            any = true;
            step = std::min<uint64_t>(step, end[i] - m->t);
            auto it = std::upper_bound(m->meas.begin(), m->meas.end(), m->t);
            if (it != m->meas.end())
                step = std::min<uint64_t>(step, *it - m->t);
        }
        if (!any)
            break;
        rc = run_sweeps(b, step);
        if (rc != EA_OK)
            return rc;
        std::vector<ea_ctx *> due;
        for (size_t i = 0; i < b->members.size(); ++i) {
            ea_ctx *m = b->members[i];
            const uint64_t adv = std::min<uint64_t>(step, end[i] - m->t);
            if (adv == 0)
                continue;
            m->t += adv;
            if (idx_of(m->meas, m->t) >= 0)
                due.push_back(m);
        }
        // each member's measurements read the state the sweeps left and write
        // the member's own sums only: given side streams, they run side by
        // side, forked from the batch stream and joined back before the next
        // sweeps
        const int lanes = b->have_side && due.size() >= 2
                              ? (int)std::min<size_t>(due.size(), 1 + ea::kSideStreams)
                              : 1;
        if (lanes > 1) {
            EA_BCUDA(b, cudaEventRecord(b->side.fork, b->stream));
            for (int r = 1; r < lanes; ++r)
                EA_BCUDA(b, cudaStreamWaitEvent(b->side.stream[r - 1], b->side.fork, 0));
        }
        for (size_t k = 0; k < due.size(); ++k) {
            const int lane = (int)(k % (size_t)lanes);
            rc = fire_measurements(due[k], lane == 0 ? b->stream : b->side.stream[lane - 1]);
            if (rc != EA_OK)
                return bfail(b, rc, "measurement failed: " + due[k]->err);
        }
        if (lanes > 1) {
            for (int r = 1; r < lanes; ++r) {
                EA_BCUDA(b, cudaEventRecord(b->side.join[r - 1], b->side.stream[r - 1]));
                EA_BCUDA(b, cudaStreamWaitEvent(b->stream, b->side.join[r - 1], 0));
            }
        }
        remaining -= step;
    }
    return EA_OK;
}

}  // namespace

extern "C" {

int ea_batch_sweep(ea_batch *b, uint64_t n)
{
    NvtxRange nvtx_range("ea_batch_sweep");
    if (!b)
        return EA_ERR_INVALID_ARG;
    return batch_sweep_impl(b, n, nullptr);
}

namespace {

// Copies of the members' spins and times, so that trial sweeps (tuning,
// profiling) leave the jobs exactly as they were.
struct SavedState {
    std::vector<uint32_t *> spins;
    std::vector<uint64_t> times;
};

int save_state(ea_batch *b, SavedState &st)
{
    st.spins.assign(b->members.size(), nullptr);
    st.times.assign(b->members.size(), 0);
    for (size_t i = 0; i < b->members.size(); ++i) {
        ea_ctx *m = b->members[i];
        st.times[i] = m->t;
        st.spins[i] = (uint32_t *)dev_alloc(m->spins_bytes, b->stream);
        if (!st.spins[i])
            return bfail(b, EA_ERR_OOM, "scratch allocation failed");
        EA_BCUDA(b, cudaMemcpyAsync(st.spins[i], m->spins, m->spins_bytes,
                                    cudaMemcpyDeviceToDevice, b->stream));
    }
    return EA_OK;
}

int restore_state(ea_batch *b, SavedState &st, int rc)
{
    for (size_t i = 0; i < st.spins.size(); ++i) {
        ea_ctx *m = b->members[i];
        m->t = st.times[i];
        if (st.spins[i] &&
            cudaMemcpyAsync(m->spins, st.spins[i], m->spins_bytes, cudaMemcpyDeviceToDevice,
                            b->stream) != cudaSuccess &&
            rc == EA_OK)
            rc = bfail(b, EA_ERR_CUDA, "state restore failed");
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && rc == EA_OK)
        rc = bfail(b, EA_ERR_CUDA, "stream synchronisation failed");
    for (size_t i = 0; i < st.spins.size(); ++i)
        dev_free(st.spins[i], b->members[i]->spins_bytes, b->stream);
    st.spins.clear();
    return rc;
}

}  // namespace

int ea_batch_profile(ea_batch *b, int sweeps, uint64_t out[4])
{
    if (!b || !out || sweeps < 1)
        return EA_ERR_INVALID_ARG;
    std::memset(out, 0, 4 * sizeof(uint64_t));
    if (b->members.empty())
        return EA_OK;
    SavedState st;
    int rc = save_state(b, st);
    unsigned long long *ctr = nullptr;
    if (rc == EA_OK) {
        ctr = (unsigned long long *)dev_alloc(4 * sizeof(unsigned long long), b->stream);
        if (!ctr)
            rc = bfail(b, EA_ERR_OOM, "counter allocation failed");
        else if (cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), b->stream) != cudaSuccess)
            rc = bfail(b, EA_ERR_CUDA, "counter reset failed");
    }
    if (rc == EA_OK)
        rc = upload_tables(b, (uint64_t)sweeps);
    if (rc == EA_OK)
        rc = enqueue_direct(b, (uint64_t)sweeps, ctr);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (rc == EA_OK &&
        (cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
         cudaStreamSynchronize(b->stream) != cudaSuccess))
        rc = bfail(b, EA_ERR_CUDA, "counter read-back failed");
    rc = restore_state(b, st, rc);
    dev_free(ctr, 4 * sizeof(unsigned long long), b->stream);
    if (rc != EA_OK)
        return rc;
    uint64_t flips = 0;
    for (ea_ctx *m : b->members)
        flips += (uint64_t)sweeps * 2ull * (uint64_t)m->S * (uint64_t)m->L * m->L * m->L;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = flips;
    return EA_OK;
}

int ea_batch_set_streams(ea_batch *b, int streams)
{
    if (!b || streams < 1 || streams > 1 + ea::kSideStreams)
        return EA_ERR_INVALID_ARG;
    b->streams = streams;
    drop_graph(b);
    return EA_OK;
}

int ea_batch_get_streams(const ea_batch *b, int *streams)
{
    if (!b || !streams)
        return EA_ERR_INVALID_ARG;
    *streams = b->streams;
    return EA_OK;
}

int ea_batch_set_resident(ea_batch *b, int max_side)
{
    if (!b || max_side < 0)
        return EA_ERR_INVALID_ARG;
    b->res_max_L = max_side;
    drop_graph(b);
    return EA_OK;
}

int ea_batch_get_resident(const ea_batch *b, int *max_side)
{
    if (!b || !max_side)
        return EA_ERR_INVALID_ARG;
    *max_side = b->res_max_L;
    return EA_OK;
}

int ea_batch_set_variant(ea_batch *b, int variant)
{
    if (!b || variant < 0 || variant > 1)
        return EA_ERR_INVALID_ARG;
    b->variant = variant;
    drop_graph(b);
    return EA_OK;
}

int ea_batch_get_variant(const ea_batch *b, int *variant)
{
    if (!b || !variant)
        return EA_ERR_INVALID_ARG;
    *variant = b->variant;
    return EA_OK;
}

int ea_batch_autotune(ea_batch *b, int trial_sweeps)
{
    NvtxRange nvtx_range("ea_batch_autotune");
    if (!b || trial_sweeps < 1)
        return EA_ERR_INVALID_ARG;
    if (b->members.empty())
        return EA_OK;
    // tuning runs on the members' state and puts it back
    SavedState st;
    int rc = save_state(b, st);
    const int cpts[3] = {1, 2, 4};
    const int graphs[3] = {0, 16, 64};
    // the sample-resident kernel is a candidate when a Metropolis member fits
    bool any_res = false;
    for (ea_ctx *m : b->members)
        any_res = any_res || (m->rule == EA_RULE_METROPOLIS && ea::res_side_fits(m->L));
    const int res_opts[3] = {ea::kResDefaultMaxL, ea::kResMaxL, 0};
    const int n_res = any_res ? 3 : 1;
    // and the staged kernel against the register-window tiles at side 128
    bool any_128 = false;
    for (ea_ctx *m : b->members)
        any_128 = any_128 || (m->rule == EA_RULE_METROPOLIS && m->L == 128);
    const int var_opts[2] = {0, 1};
    const int n_var = any_128 ? 2 : 1;
    // and the number of streams, given side streams and two or more members
    const int str_opts[4] = {1, 2, 3, 4};
    const int n_str = b->have_side && b->members.size() >= 2 ? 4 : 1;
    float best = 1e30f;
    int best_cpt = b->cpt, best_graph = b->graph_sweeps, best_res = b->res_max_L;
    int best_var = b->variant, best_str = b->streams;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == EA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bfail(b, EA_ERR_CUDA, "event creation failed");
    for (int si = 0; si < n_str && rc == EA_OK; ++si)
    for (int vi = 0; vi < n_var && rc == EA_OK; ++vi)
    for (int ri = 0; ri < n_res && rc == EA_OK; ++ri)
    for (int ci = 0; ci < 3 && rc == EA_OK; ++ci) {
        for (int gi = 0; gi < 3 && rc == EA_OK; ++gi) {
            if (graphs[gi] > 0 && b->stream == nullptr)
                continue;
            b->res_max_L = any_res ? res_opts[ri] : b->res_max_L;
            b->variant = any_128 ? var_opts[vi] : b->variant;
            b->streams = n_str > 1 ? str_opts[si] : b->streams;
            b->cpt = cpts[ci];
            b->graph_sweeps = graphs[gi] > 0 ? std::min(graphs[gi], trial_sweeps) : 0;
            rc = upload_tables(b, ea::kMaxTime);
            if (rc == EA_OK)
                rc = run_sweeps(b, (uint64_t)b->graph_sweeps > 0 ? b->graph_sweeps : 1);  // warm
            if (rc != EA_OK)
                break;
            cudaEventRecord(e0, b->stream);
            rc = run_sweeps(b, (uint64_t)trial_sweeps);
            cudaEventRecord(e1, b->stream);
            if (rc != EA_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = rc != EA_OK ? rc : bfail(b, EA_ERR_CUDA, "autotune timing failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_cpt = b->cpt;
                best_graph = b->graph_sweeps;
                best_res = b->res_max_L;
                best_var = b->variant;
                best_str = b->streams;
            }
        }
    }
    rc = restore_state(b, st, rc);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    b->cpt = best_cpt;
    b->graph_sweeps = best_graph;
    b->res_max_L = best_res;
    b->variant = best_var;
    b->streams = best_str;
    drop_graph(b);
    return rc;
}

int ea_batch_destroy(ea_batch *b)
{
    if (!b)
        return EA_OK;
    cudaStreamSynchronize(b->stream);
    for (ea_ctx *m : b->members) {
        m->batch = nullptr;
        m->stream = m->own_stream;
    }
    drop_graph(b);
    for (int r = 0; r < 2; ++r) {
        dev_free(b->tab_dev[r], b->cap[r] * sizeof(ea::JobDev), b->stream);
    }
    for (int i = 0; i < ea::kSideStreams; ++i) {
        if (b->side.stream[i])
            cudaStreamDestroy(b->side.stream[i]);
        if (b->side.join[i])
            cudaEventDestroy(b->side.join[i]);
    }
    if (b->side.fork)
        cudaEventDestroy(b->side.fork);
    delete b;
    return EA_OK;
}

const char *ea_batch_last_error(const ea_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// serving
// ---------------------------------------------------------------------------
namespace {

struct ServerJob {
    int64_t id = 0;
    ea_job_spec spec;
    std::vector<uint64_t> tw, tt;
    int state = EA_JOB_QUEUED;
    ea_ctx *ctx = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct ea_server {
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    int max_running = 0;
    uint64_t chunk = 0;
    ea_batch *batch = nullptr;
    std::deque<ServerJob *> queue;
    std::vector<ServerJob *> running;
    std::map<int64_t, ServerJob *> jobs;
    size_t in_use = 0;
    int64_t next_id = 1;
    uint64_t flips = 0;
    uint64_t steps = 0;
    std::string err;
};

namespace {

int sfail(ea_server *srv, int code, const std::string &msg)
{
    if (srv)
        srv->err = msg;
    return code;
}

// Create, schedule and quench the job's context on the server's stream.
int start_job(ea_server *srv, ServerJob *j)
{
    const ea_job_spec &sp = j->spec;
    ea_ctx *c = nullptr;
    int rc = ea_create_samples(&c, sp.L, sp.p_neg, sp.seed, sp.n_samples, sp.rng_group_G,
                               (void *)srv->stream);
    if (rc != EA_OK)
        return rc;
    rc = ea_set_schedule(c, j->tw.data(), (int)j->tw.size(), j->tt.data(), (int)j->tt.size());
    if (rc == EA_OK)
        rc = ea_quench(c, sp.T, sp.rule);
    if (rc == EA_OK)
        rc = ea_batch_add(srv->batch, c);
    if (rc != EA_OK) {
        ea_destroy(c);
        return rc;
    }
    j->ctx = c;
    return EA_OK;
}

}  // namespace

extern "C" {

int ea_server_create(ea_server **out, size_t budget_bytes, int max_running, uint64_t chunk_sweeps,
                     void *cuda_stream)
{
    if (!out || max_running < 1 || chunk_sweeps == 0 || chunk_sweeps > ea::kMaxTime)
        return EA_ERR_INVALID_ARG;
    *out = nullptr;
    ea_server *srv = new (std::nothrow) ea_server();
    if (!srv)
        return EA_ERR_OOM;
    srv->stream = (cudaStream_t)cuda_stream;
    srv->budget = budget_bytes;
    srv->max_running = max_running;
    srv->chunk = chunk_sweeps;
    const int rc = ea_batch_create(&srv->batch, cuda_stream);
    if (rc != EA_OK) {
        delete srv;
        return rc;
    }
    // launch shape of the running set: 4 word columns per thread and, off the
    // legacy stream, 16-sweep graphs (the shape the autotuner picks for large
    // lattices); ea_server_configure changes it
    ea_batch_configure(srv->batch, 4, cuda_stream ? 16 : 0);
    *out = srv;
    return EA_OK;
}

int ea_server_submit(ea_server *srv, const ea_job_spec *spec, int64_t *job_id)
{
    if (!srv || !spec || !job_id)
        return EA_ERR_INVALID_ARG;
    Geo g;
    if (ea::make_geo(spec->L, &g) != 0 || !(spec->p_neg >= 0.0 && spec->p_neg <= 1.0) ||
        spec->n_samples < 1 || spec->n_samples > ea::kMaxSamples || spec->rng_group_G < 1 ||
        !(spec->T >= 0.0) || (spec->rule != EA_RULE_METROPOLIS && spec->rule != EA_RULE_HEATBATH) ||
        spec->sweeps >= ea::kMaxTime || spec->n_tw < 0 || spec->n_t < 0 ||
        spec->n_tw > ea::kMaxSchedule || spec->n_t > ea::kMaxSchedule ||
        (spec->n_tw > 0 && !spec->t_w) || (spec->n_t > 0 && !spec->t))
        return sfail(srv, EA_ERR_INVALID_ARG, "invalid job spec");
    ServerJob *j = new (std::nothrow) ServerJob();
    if (!j)
        return EA_ERR_OOM;
    j->spec = *spec;
    j->tw.assign(spec->t_w, spec->t_w + spec->n_tw);
    j->tt.assign(spec->t, spec->t + spec->n_t);
    j->spec.t_w = nullptr;
    j->spec.t = nullptr;
    if (ea_footprint(spec->L, spec->n_samples, spec->n_tw, spec->n_t, &j->bytes) != EA_OK ||
        j->bytes > srv->budget) {
        delete j;
        return sfail(srv, EA_ERR_INVALID_ARG, "job footprint exceeds the server budget");
    }
    j->id = srv->next_id++;
    srv->jobs[j->id] = j;
    srv->queue.push_back(j);
    *job_id = j->id;
    return EA_OK;
}

int ea_server_step(ea_server *srv, int *n_finished)
{
    NvtxRange nvtx_range("ea_server_step");
    if (!srv)
        return EA_ERR_INVALID_ARG;
    if (n_finished)
        *n_finished = 0;
    // 1. admission, first fit in submission order
    for (auto it = srv->queue.begin(); it != srv->queue.end();) {
        ServerJob *j = *it;
        if ((int)srv->running.size() >= srv->max_running)
            break;
        if (srv->in_use + j->bytes > srv->budget) {
            ++it;
            continue;
        }
        const int rc = start_job(srv, j);
        if (rc == EA_ERR_OOM) {
            ++it;  // the device is fuller than the budget says: try again later
            continue;
        }
        if (rc != EA_OK)
            return sfail(srv, rc, "job admission failed");
        srv->in_use += j->bytes;
        j->state = EA_JOB_RUNNING;
        srv->running.push_back(j);
        it = srv->queue.erase(it);
    }
    if (srv->running.empty())
        return EA_OK;
    // 2. one chunk for every running job, each stopping at its own sweep count
    std::vector<uint64_t> limits;
    for (ea_ctx *m : srv->batch->members) {
        ServerJob *owner = nullptr;
        for (ServerJob *j : srv->running)
            if (j->ctx == m)
                owner = j;
        limits.push_back(owner ? owner->spec.sweeps - m->t : 0);
    }
    std::vector<uint64_t> before;
    for (ServerJob *j : srv->running)
        before.push_back(j->ctx->t);
    int rc = batch_sweep_impl(srv->batch, srv->chunk, &limits);
    if (rc != EA_OK)
        return sfail(srv, rc, "batch sweep failed: " + srv->batch->err);
    ++srv->steps;
    // 3. retire
    std::vector<ServerJob *> still;
    for (size_t i = 0; i < srv->running.size(); ++i) {
        ServerJob *j = srv->running[i];
        const uint64_t N = (uint64_t)j->spec.L * j->spec.L * j->spec.L;
        srv->flips += (j->ctx->t - before[i]) * 2ull * (uint64_t)j->spec.n_samples * N;
        if (j->ctx->t >= j->spec.sweeps) {
            ea_batch_remove(srv->batch, j->ctx);
            j->state = EA_JOB_DONE;
            if (n_finished)
                ++*n_finished;
        } else {
            still.push_back(j);
        }
    }
    srv->running.swap(still);
    return EA_OK;
}

int ea_server_configure(ea_server *srv, int cols_per_thread, int graph_sweeps)
{
    if (!srv)
        return EA_ERR_INVALID_ARG;
    return ea_batch_configure(srv->batch, cols_per_thread, graph_sweeps);
}

int ea_server_job_state(const ea_server *srv, int64_t job_id, int *state, uint64_t *time)
{
    if (!srv || !state)
        return EA_ERR_INVALID_ARG;
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end())
        return EA_ERR_INVALID_ARG;
    *state = it->second->state;
    if (time)
        *time = it->second->ctx ? it->second->ctx->t : 0;
    return EA_OK;
}

int ea_server_job(ea_server *srv, int64_t job_id, ea_ctx **job)
{
    if (!srv || !job)
        return EA_ERR_INVALID_ARG;
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end())
        return EA_ERR_INVALID_ARG;
    if (!it->second->ctx)
        return sfail(srv, EA_ERR_STATE, "job still queued");
    *job = it->second->ctx;
    return EA_OK;
}

int ea_server_release(ea_server *srv, int64_t job_id)
{
    if (!srv)
        return EA_ERR_INVALID_ARG;
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end())
        return EA_ERR_INVALID_ARG;
    ServerJob *j = it->second;
    if (j->state != EA_JOB_DONE)
        return sfail(srv, EA_ERR_STATE, "job not done");
    ea_destroy(j->ctx);
    srv->in_use -= j->bytes;
    srv->jobs.erase(it);
    delete j;
    return EA_OK;
}

int ea_server_cancel(ea_server *srv, int64_t job_id)
{
    if (!srv)
        return EA_ERR_INVALID_ARG;
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end())
        return sfail(srv, EA_ERR_INVALID_ARG, "unknown job");
    ServerJob *j = it->second;
    if (j->state == EA_JOB_QUEUED) {
        srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), j));
    } else if (j->state == EA_JOB_RUNNING) {
        ea_batch_remove(srv->batch, j->ctx);
        srv->running.erase(std::find(srv->running.begin(), srv->running.end(), j));
    }
    if (j->ctx) {
        ea_destroy(j->ctx);
        srv->in_use -= j->bytes;
    }
    srv->jobs.erase(it);
    delete j;
    return EA_OK;
}

int ea_server_get_stats(const ea_server *srv, ea_server_stats *out)
{
    if (!srv || !out)
        return EA_ERR_INVALID_ARG;
    out->queued = (int)srv->queue.size();
    out->running = (int)srv->running.size();
    out->done = (int)(srv->jobs.size() - srv->queue.size() - srv->running.size());
    out->bytes_in_use = srv->in_use;
    out->flips = srv->flips;
    out->steps = srv->steps;
    return EA_OK;
}

int ea_server_destroy(ea_server *srv)
{
    if (!srv)
        return EA_OK;
    ea_batch_destroy(srv->batch);
    for (auto &kv : srv->jobs) {
        ea_destroy(kv.second->ctx);
        delete kv.second;
    }
    delete srv;
    return EA_OK;
}

const char *ea_server_last_error(const ea_server *srv) { return srv ? srv->err.c_str() : ""; }

}  // extern "C"
