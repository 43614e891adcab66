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
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ea_ageing.h"
#include "ea_internal.h"

using ea::Geo;

namespace {

ea_alloc_fn g_alloc = nullptr;
ea_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;

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

static ea::Thr make_thr(int rule, const uint64_t thr_k[7], const uint8_t always_k[7])
{
    ea::Thr t;
    std::memset(&t, 0, sizeof(t));
    t.rule = rule;
    int n_always = 0;
    for (int u = 0; u < 7; ++u) {
        // u unsatisfied bonds <=> dE = 12 - 4u <=> k = 6 - u
        t.thr_u[u] = thr_k[6 - u];
        if (always_k[6 - u]) {
            t.always_u |= 1u << u;
            ++n_always;
        }
    }
    t.all_always = n_always == 7;
    // lanes that compare a random number: every u not accepted outright
    bool any_nonzero = false;
    uint32_t zero_calls = 0;
    const int nu = rule == EA_RULE_METROPOLIS ? 3 : 7;
    for (int call = 0; call < 16; ++call) {
        bool zero = true;
        for (int u = 0; u < nu; ++u) {
            if ((t.always_u >> u) & 1u)
                continue;
            const uint64_t nib = (t.thr_u[u] >> (60 - 4 * call)) & 0xFu;
            if (nib)
                zero = false;
        }
        if (zero)
            zero_calls |= 1u << call;
    }
    for (int u = 0; u < nu; ++u)
        if (!((t.always_u >> u) & 1u) && t.thr_u[u] != 0)
            any_nonzero = true;
    t.zero_calls = zero_calls;
    // with every needed threshold 0 no lane can accept: skip the random numbers
    t.none_random = !any_nonzero;
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
    int G = 1;
    cudaStream_t stream = nullptr;
    Geo geo;

    uint32_t *spins = nullptr;
    uint32_t *J = nullptr;
    uint32_t *snaps = nullptr;
    unsigned long long *res = nullptr;
    size_t spins_bytes = 0, J_bytes = 0, snaps_bytes = 0, res_bytes = 0;

    std::vector<uint64_t> tw, tt, meas;
    size_t off_q = 0, off_u = 0, off_g = 0, off_a = 0;  // in counters

    bool quenched = false;
    double T = 0;
    int rule = 0;
    uint64_t thr_k[7] = {0};
    uint8_t always_k[7] = {0};
    ea::Thr thr;
    uint64_t t = 0;

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

ea::SweepLaunch sweep_args(const ea_ctx *c)
{
    ea::SweepLaunch p;
    p.spins = c->spins;
    p.J = c->J;
    p.geo = c->geo;
    p.thr = c->thr;
    p.key0 = (uint32_t)c->seed;
    p.key1 = (uint32_t)(c->seed >> 32);
    p.n_samples = c->S;
    p.rng_group = c->G;
    return p;
}

// Measurements due at the current time c->t (if it is a scheduled time).
int fire_measurements(ea_ctx *c)
{
    const int mi = idx_of(c->meas, c->t);
    if (mi < 0)
        return EA_OK;
    const size_t S = (size_t)c->S, R = (size_t)c->R();
    const size_t area = c->area_words();
    EA_CUDA(c, ea::launch_obs_state(c->spins, c->J, c->geo, c->S, c->res + c->off_q + mi * S,
                                    c->res + c->off_u + mi * S * 2, c->stream));
    const int ti = idx_of(c->tw, c->t);
    if (ti >= 0) {
        EA_CUDA(c, cudaMemcpyAsync(c->snaps + ti * area, c->spins, area * sizeof(uint32_t),
                                   cudaMemcpyDeviceToDevice, c->stream));
        EA_CUDA(c, ea::launch_obs_c4(c->spins, c->geo, c->S, c->res + c->off_g + ti * S * 3 * R,
                                     c->stream));
    }
    for (size_t i = 0; i < c->tw.size() && c->tw[i] <= c->t; ++i) {
        const int j = idx_of(c->tt, c->t - c->tw[i]);
        if (j < 0)
            continue;
        const size_t slot = c->off_a + (i * c->tt.size() + (size_t)j) * S * 2;
        EA_CUDA(c, ea::launch_obs_autocorr(c->snaps + i * area, c->spins, c->geo, c->S,
                                           c->res + slot, c->stream));
    }
    return EA_OK;
}

int check_ctx(const ea_ctx *c) { return c ? EA_OK : EA_ERR_INVALID_ARG; }

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
    if (!out)
        return EA_ERR_INVALID_ARG;
    *out = nullptr;
    Geo g;
    if (ea::make_geo(L, &g) != 0 || !(p_neg >= 0.0 && p_neg <= 1.0) || n_samples < 1 ||
        n_samples > ea::kMaxSamples || rng_group_G < 1)
        return EA_ERR_INVALID_ARG;
    ea_ctx *c = new (std::nothrow) ea_ctx();
    if (!c)
        return EA_ERR_OOM;
    c->L = L;
    c->p_neg = p_neg;
    c->seed = seed;
    c->S = n_samples;
    c->G = rng_group_G;
    c->stream = (cudaStream_t)cuda_stream;
    c->geo = g;
    c->spins_bytes = c->area_words() * sizeof(uint32_t);
    c->J_bytes = (size_t)n_samples * 3 * g.words * sizeof(uint32_t);
    c->spins = (uint32_t *)dev_alloc(c->spins_bytes, c->stream);
    c->J = (uint32_t *)dev_alloc(c->J_bytes, c->stream);
    if (!c->spins || !c->J) {
        ea_destroy(c);
        return EA_ERR_OOM;
    }
    cudaError_t e = ea::launch_init_couplings(c->J, g, n_samples, p_neg, seed, c->stream);
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
    c->thr = make_thr(rule, thr, alw);
    EA_CUDA(c, ea::launch_init_spins(c->spins, c->geo, c->S, c->seed, c->stream));
    if (c->res)
        EA_CUDA(c, cudaMemsetAsync(c->res, 0, c->res_bytes, c->stream));
    c->t = 0;
    c->quenched = true;
    return fire_measurements(c);
}

int ea_sweep(ea_ctx *c, uint64_t n)
{
    if (check_ctx(c))
        return EA_ERR_INVALID_ARG;
    if (!c->quenched)
        return fail(c, EA_ERR_STATE, "ea_sweep before ea_quench");
    if (n > ea::kMaxTime || c->t + n > ea::kMaxTime)
        return fail(c, EA_ERR_INVALID_ARG, "time would pass 2^48");
    const uint64_t target = c->t + n;
    const ea::SweepLaunch p = sweep_args(c);
    while (c->t < target) {
        auto it = std::upper_bound(c->meas.begin(), c->meas.end(), c->t);
        const uint64_t stop = (it == c->meas.end()) ? target : std::min(target, *it);
        EA_CUDA(c, ea::launch_sweeps(p, c->t, stop - c->t, c->stream));
        c->t = stop;
        const int rc = fire_measurements(c);
        if (rc != EA_OK)
            return rc;
    }
    return EA_OK;
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
    std::vector<unsigned long long> a(S * 2), q(S), u(S * 2), gp(S * 3 * R);
    const size_t slot_a = c->off_a + ((size_t)i * c->tt.size() + (size_t)j) * S * 2;
    EA_CUDA(c, cudaMemcpyAsync(a.data(), c->res + slot_a, a.size() * 8, cudaMemcpyDeviceToHost,
                               c->stream));
    EA_CUDA(c, cudaMemcpyAsync(q.data(), c->res + c->off_q + mi * S, q.size() * 8,
                               cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaMemcpyAsync(u.data(), c->res + c->off_u + mi * S * 2, u.size() * 8,
                               cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaMemcpyAsync(gp.data(), c->res + c->off_g + (size_t)i * S * 3 * R,
                               gp.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    EA_CUDA(c, cudaStreamSynchronize(c->stream));

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
constexpr char kMagic[8] = {'E', 'A', 'G', 'B', '3', '0', '0', '\1'};

struct CkptHeader {
    char magic[8];
    int32_t L, S, G, rule;
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
    int rc = ea_create_samples(&c, h.L, h.p_neg, h.seed, h.S, h.G, cuda_stream);
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
            c->thr = make_thr(h.rule, thr, alw);
        }
    }
    if (rc == EA_OK) {
        bool ok = read_dev(f, c->spins, c->spins_bytes, c->stream) &&
                  read_dev(f, c->J, c->J_bytes, c->stream) &&
                  read_dev(f, c->snaps, c->snaps_bytes, c->stream) &&
                  read_dev(f, c->res, c->res_bytes, c->stream);
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
    *out = c;
    return EA_OK;
}

int ea_destroy(ea_ctx *c)
{
    if (!c)
        return EA_OK;
    if (c->spins || c->J || c->snaps || c->res)
        cudaStreamSynchronize(c->stream);
    release_schedule(c);
    dev_free(c->spins, c->spins_bytes, c->stream);
    dev_free(c->J, c->J_bytes, c->stream);
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
