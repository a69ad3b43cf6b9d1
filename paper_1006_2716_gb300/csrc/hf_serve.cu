// hf_serve.cu -- continuously batched impurity-solve service (C ABI in include/hf.h).
//
// In real-space DMFT every inequivalent site of every run needs one Hirsch-Fye impurity solve
// per self-consistency iteration ("Model and Methods": the impurity problems are independent
// and local in the site index).  This service accepts such solves as requests from any host
// thread and runs them on one GPU:
//   * a scheduler thread in the library admits queued requests in arrival order as device memory
//     frees up -- each needs chains x (2 L^2 Green-function entries + fields + bins), carved
//     first-fit out of a caller-owned device pool -- and as one of its streams frees up;
//   * up to 16 admitted requests share one launch of the fused sweep kernel; several launches
//     run concurrently on separate streams, so requests that arrive while others are on the GPU
//     start without waiting for them (continuous batching);
//   * the Ising fields and sweep counters of every (run, site) key stay on the device between
//     requests as warm starts; a key's next request waits until its previous one completes.
// Each chain is computed exactly as in a context of its own, so a result does not depend on
// which other requests shared its launch.  All waits are host-side and non-blocking; nothing on
// the device polls or spins.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hf_internal.cuh"

namespace {

constexpr int kMaxLServe = 64;
constexpr int kMaxPerLaunch = hfk::kMaxProblems;
using Clock = std::chrono::steady_clock;

thread_local std::string g_srv_error;

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// First-fit allocator over [0, size) with coalescing of freed ranges.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        n = align256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align256(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Job {
    uint64_t ticket = 0;
    hf_request req{};
    Clock::time_point t_submit;
    // device placement while admitted
    size_t off = 0, bytes = 0;
    int key = -1;
    bool warm = false;
};

struct Launch {
    std::vector<Job> jobs;
    int stream = 0;
    cudaEvent_t done = nullptr;
};

// Per-request device layout inside its arena block.
struct Block {
    double* gtau;      // [2][L]
    double* g0inv;     // [2][L*L] inverse bath matrices of the refreshes
    double* G;         // [cps][2][L*L]
    int8_t* s;         // [cps][L]
    uint32_t* nsw;     // [cps]
    uint32_t* nmeas;   // [cps]
    unsigned long long* acc;  // [cps]
    double* bins;      // [cps][nb][2L+3]
    double* obs;       // [2][2L+4]  mean, err
    int* status;       // [4]
};

}  // namespace

struct hf_srv {
    hf_srv_params p{};
    int nb = 0;                      // bins per solve
    int device = 0;
    char* pool = nullptr;            // caller's device pool
    size_t pool_bytes = 0;
    // warm-start store: per key, fields [cps][max_L] and counters [cps]
    int8_t* warm_s = nullptr;
    uint32_t* warm_nsw = nullptr;
    size_t arena_off = 0;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    // pinned host staging: per stream, up to kMaxPerLaunch requests
    double* h_in = nullptr;          // [nstreams][kMaxPerLaunch][2][kMaxLServe]
    double* h_out = nullptr;         // [nstreams][kMaxPerLaunch][2][2*kMaxLServe+4]
    uint32_t* h_cnt = nullptr;       // [nstreams][kMaxPerLaunch]
    // keys
    std::map<std::pair<int, int>, int> key_of;
    std::vector<int> key_busy;       // 1 while a request of the key is admitted
    std::vector<int> key_valid;      // 1 once the key holds fields
    std::vector<int> key_L;          // L of the fields the key holds (its last request's L)
    std::vector<uint64_t> key_used;  // LRU clock
    uint64_t lru_clock = 0;
    // queues and results
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job> queue;
    std::vector<Launch> inflight;
    std::unordered_map<uint64_t, hf_result> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    int peak_inflight = 0;
    size_t peak_bytes = 0;
    uint64_t n_completed = 0;
    std::string err;
    std::thread worker;
};

namespace {

hf_status sfail(hf_srv* s, hf_status st, const std::string& m) {
    if (st == HF_ECUDA) (void)cudaGetLastError();
    if (s) s->err = m; else g_srv_error = m;
    return st;
}

int L_of(const hf_request& r) { return r.L; }

size_t job_bytes(const hf_srv_params& p, int nb, int L) {
    const size_t cps = static_cast<size_t>(p.chains_per_request);
    size_t n = 0;
    n += align256(sizeof(double) * 2 * L);
    n += align256(sizeof(double) * 2 * L * L);
    n += align256(sizeof(double) * cps * 2 * L * L);
    n += align256(cps * L);
    n += align256(sizeof(uint32_t) * cps) * 2;
    n += align256(sizeof(unsigned long long) * cps);
    n += align256(sizeof(double) * cps * nb * (2 * L + 3));
    n += align256(sizeof(double) * 2 * (2 * L + 4));
    n += align256(sizeof(int) * 4);
    return n;
}

Block carve(char* base, const hf_srv_params& p, int nb, int L) {
    const size_t cps = static_cast<size_t>(p.chains_per_request);
    Block b{};
    size_t o = 0;
    auto take = [&](size_t n) { char* q = base + o; o += align256(n); return q; };
    b.gtau = reinterpret_cast<double*>(take(sizeof(double) * 2 * L));
    b.g0inv = reinterpret_cast<double*>(take(sizeof(double) * 2 * L * L));
    b.G = reinterpret_cast<double*>(take(sizeof(double) * cps * 2 * L * L));
    b.s = reinterpret_cast<int8_t*>(take(cps * L));
    b.nsw = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * cps));
    b.nmeas = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * cps));
    b.acc = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * cps));
    b.bins = reinterpret_cast<double*>(take(sizeof(double) * cps * nb * (2 * L + 3)));
    b.obs = reinterpret_cast<double*>(take(sizeof(double) * 2 * (2 * L + 4)));
    b.status = reinterpret_cast<int*>(take(sizeof(int) * 4));
    return b;
}

size_t warm_bytes(const hf_srv_params& p) {
    const size_t cps = static_cast<size_t>(p.chains_per_request);
    return align256(cps * p.max_L * p.max_keys) + align256(sizeof(uint32_t) * cps * p.max_keys);
}

hf_status validate_srv(const hf_srv_params* p, std::string& e) {
    if (!p) { e = "null params"; return HF_EINVAL; }
    if (p->chains_per_request < 1 || p->chains_per_request > 4096) { e = "chains_per_request out of range"; return HF_EINVAL; }
    if (p->n_warmup < 0 || p->n_measure < 1) { e = "need n_warmup >= 0 and n_measure >= 1"; return HF_EINVAL; }
    if (p->bin_size < 1 || p->n_measure % p->bin_size != 0) { e = "n_measure must be a multiple of bin_size"; return HF_EINVAL; }
    if (p->refresh_every < 0) { e = "refresh_every must be >= 0"; return HF_EINVAL; }
    if (p->refresh_stagger != 0 && p->refresh_stagger != 1) { e = "refresh_stagger must be 0 or 1"; return HF_EINVAL; }
    if (p->precision != 0 && p->precision != 2) { e = "precision must be 0 (FP64) or 2 (FP32 pairs)"; return HF_EINVAL; }
    if (!hfk::qmc_f64_supported(p->max_L)) { e = "max_L must be one of 8,12,16,20,24,32,40,48,64"; return HF_EINVAL; }
    if (p->max_keys < 1 || p->n_streams < 1 || p->n_streams > 64) { e = "max_keys >= 1 and 1 <= n_streams <= 64 required"; return HF_EINVAL; }
    if (p->max_inflight < 1) { e = "max_inflight must be >= 1"; return HF_EINVAL; }
    if (!(p->team_warps == 0 || p->team_warps == 1 || p->team_warps == 2 || p->team_warps == 4)) { e = "team_warps must be 0, 1, 2 or 4"; return HF_EINVAL; }
    return HF_OK;
}

// Starts one launch with the admitted jobs on stream si (caller holds no lock; jobs are owned).
hf_status start_launch(hf_srv* S, Launch& Lh) {
    const int si = Lh.stream;
    cudaStream_t st = S->streams[si];
    const hf_srv_params& p = S->p;
    const int cps = p.chains_per_request;
    hfk::QmcBatch qb{};
    qb.nprob = static_cast<int>(Lh.jobs.size());
    size_t smem = 0;
    int blocks = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < qb.nprob && e == cudaSuccess; ++k) {
        Job& j = Lh.jobs[k];
        const int L = L_of(j.req);
        Block b = carve(S->pool + S->arena_off + j.off, p, S->nb, L);
        double* hin = S->h_in + (static_cast<size_t>(si) * kMaxPerLaunch + k) * 2 * kMaxLServe;
        std::memcpy(hin, j.req.g0_tau[0], sizeof(double) * L);
        std::memcpy(hin + L, j.req.g0_tau[1], sizeof(double) * L);
        e = cudaMemcpyAsync(b.gtau, hin, sizeof(double) * 2 * L, cudaMemcpyHostToDevice, st);
        int8_t* ws = S->warm_s + static_cast<size_t>(j.key) * cps * p.max_L;
        uint32_t* wn = S->warm_nsw + static_cast<size_t>(j.key) * cps;
        if (e == cudaSuccess) {
            if (j.warm) {
                e = cudaMemcpy2DAsync(b.s, L, ws, p.max_L, L, cps, cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b.nsw, wn, sizeof(uint32_t) * cps, cudaMemcpyDeviceToDevice, st);
            } else {
                e = hfk::launch_init_fields(b.s, cps, cps, L, static_cast<uint32_t>(j.req.seed & 0xFFFFFFFFull),
                                            static_cast<uint32_t>(j.req.seed >> 32), st, j.req.site);
                if (e == cudaSuccess) e = cudaMemsetAsync(b.nsw, 0, sizeof(uint32_t) * cps, st);
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(b.nmeas, 0, sizeof(uint32_t) * cps, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.acc, 0, sizeof(unsigned long long) * cps, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.bins, 0, sizeof(double) * cps * S->nb * (2 * L + 3), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.status, 0, sizeof(int) * 4, st);
        // the problem of this request: one site (its key's site word), cps chains
        hfk::QmcProblem& q = qb.p[k];
        const double dtau = j.req.beta / L;
        const double lambda = std::acosh(std::exp(dtau * j.req.U / 2.0));
        q.L = L;
        q.cps = cps;
        q.nchain = cps;
        q.block0 = blocks;
        q.site0 = j.req.site;
        q.seed_lo = static_cast<uint32_t>(j.req.seed & 0xFFFFFFFFull);
        q.seed_hi = static_cast<uint32_t>(j.req.seed >> 32);
        q.a_p = std::exp(-2.0 * lambda) - 1.0;
        q.a_m = std::exp(2.0 * lambda) - 1.0;
        q.ev_p = std::exp(lambda) - 1.0;
        q.ev_m = std::exp(-lambda) - 1.0;
        q.af_p = static_cast<float>(q.a_p);
        q.af_m = static_cast<float>(q.a_m);
        q.afl_p = static_cast<float>(q.a_p - static_cast<double>(q.af_p));
        q.afl_m = static_cast<float>(q.a_m - static_cast<double>(q.af_m));
        q.n_warmup = p.n_warmup;
        q.n_measure = p.n_measure;
        q.refresh_every = p.refresh_every;
        q.refresh_stagger = p.refresh_stagger;
        q.slot_mult = 1;
        q.bin_size = p.bin_size;
        q.max_bins = S->nb;
        q.refresh_first = 1;
        q.team_warps = p.team_warps > 0 ? p.team_warps : hfk::qmc_default_team_warps(L);
        q.delay_k = 1;
        if (L > 32 && q.team_warps == 1) q.team_warps = 2;
        q.gtau = b.gtau;
        q.g0inv = b.g0inv;
        q.G = b.G;
        q.s = b.s;
        q.nsw = b.nsw;
        q.nmeas = b.nmeas;
        q.acc = b.acc;
        q.bins = b.bins;
        q.status = b.status;
        const int cpb = hfk::qmc_f64_chains_per_block(L, q.team_warps);
        blocks += (cps + cpb - 1) / cpb;
        smem = std::max(smem, p.precision == 2 ? hfk::qmc_df64_smem_bytes(L, q.team_warps, 1)
                                               : hfk::qmc_f64_smem_bytes(L, q.team_warps));
    }
    qb.nblocks = blocks;
    if (e == cudaSuccess) e = hfk::launch_g0_inverse(qb, st);   // every request brings a new bath
    if (e == cudaSuccess)
        e = (p.precision == 2) ? hfk::launch_qmc_df64(qb, smem, st) : hfk::launch_qmc_f64(qb, smem, st);
    for (int k = 0; k < qb.nprob && e == cudaSuccess; ++k) {
        Job& j = Lh.jobs[k];
        const int L = L_of(j.req);
        Block b = carve(S->pool + S->arena_off + j.off, p, S->nb, L);
        e = hfk::launch_reduce(b.bins, 1, cps, L, S->nb, S->nb, p.bin_size, b.obs, b.obs + (2 * L + 4), st);
        int8_t* ws = S->warm_s + static_cast<size_t>(j.key) * cps * p.max_L;
        uint32_t* wn = S->warm_nsw + static_cast<size_t>(j.key) * cps;
        if (e == cudaSuccess) e = cudaMemcpy2DAsync(ws, p.max_L, b.s, L, L, cps, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(wn, b.nsw, sizeof(uint32_t) * cps, cudaMemcpyDeviceToDevice, st);
        double* hout = S->h_out + (static_cast<size_t>(si) * kMaxPerLaunch + k) * 2 * (2 * kMaxLServe + 4);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hout, b.obs, sizeof(double) * 2 * (2 * L + 4), cudaMemcpyDeviceToHost, st);
        uint32_t* hc = S->h_cnt + static_cast<size_t>(si) * kMaxPerLaunch + k;
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, b.nsw, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        int* hs = reinterpret_cast<int*>(S->h_cnt + static_cast<size_t>(S->streams.size()) * kMaxPerLaunch) +
                  static_cast<size_t>(si) * kMaxPerLaunch + k;
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, b.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(Lh.done, st);
    if (e != cudaSuccess) return sfail(S, HF_ECUDA, std::string("serve launch: ") + cudaGetErrorString(e));
    return HF_OK;
}

// Completes finished launches and admits queued jobs.  Called by the scheduler thread only.
void progress(hf_srv* S) {
    const hf_srv_params& p = S->p;
    // 1. completions
    for (size_t i = 0; i < S->inflight.size();) {
        Launch& Lh = S->inflight[i];
        const cudaError_t q = cudaEventQuery(Lh.done);
        if (q == cudaErrorNotReady) { ++i; continue; }
        const auto now = Clock::now();
        std::vector<hf_result> res;
        for (size_t k = 0; k < Lh.jobs.size(); ++k) {
            const Job& j = Lh.jobs[k];
            const int L = L_of(j.req);
            hf_result r{};
            r.ticket = j.ticket;
            r.L = L;
            r.warm = j.warm ? 1 : 0;
            r.latency_s = std::chrono::duration<double>(now - j.t_submit).count();
            const int dev_status = reinterpret_cast<int*>(S->h_cnt + S->streams.size() * kMaxPerLaunch)
                [static_cast<size_t>(Lh.stream) * kMaxPerLaunch + k];
            r.status = (q != cudaSuccess) ? HF_ECUDA : (dev_status != 0 ? dev_status : HF_OK);
            if (q == cudaSuccess) {
                const double* o = S->h_out + (static_cast<size_t>(Lh.stream) * kMaxPerLaunch + k) * 2 * (2 * kMaxLServe + 4);
                std::memcpy(r.gtau[0], o, sizeof(double) * L);
                std::memcpy(r.gtau[1], o + L, sizeof(double) * L);
                r.n[0] = o[2 * L];
                r.n[1] = o[2 * L + 1];
                r.d = o[2 * L + 2];
                r.m = o[2 * L + 3];
                std::memcpy(r.err, o + (2 * L + 4), sizeof(double) * (2 * L + 4));
                r.sweeps_done = S->h_cnt[static_cast<size_t>(Lh.stream) * kMaxPerLaunch + k];
            }
            res.push_back(r);
        }
        {
            std::lock_guard<std::mutex> g(S->mu);
            for (size_t k = 0; k < Lh.jobs.size(); ++k) {
                const Job& j = Lh.jobs[k];
                S->arena.release(j.off, j.bytes);
                S->key_busy[j.key] = 0;
                S->key_valid[j.key] = (res[k].status == HF_OK) ? 1 : 0;
                S->key_L[j.key] = j.req.L;
                S->done[j.ticket] = res[k];
                ++S->n_completed;
            }
            S->stream_busy[Lh.stream] = false;
        }
        if (q != cudaSuccess && q != cudaErrorNotReady) (void)cudaGetLastError();
        cudaEventDestroy(Lh.done);
        S->inflight.erase(S->inflight.begin() + static_cast<long>(i));
        S->cv.notify_all();
    }
    // 2. admission, in arrival order, while a stream and memory are free
    while (true) {
        Launch Lh;
        {
            std::lock_guard<std::mutex> g(S->mu);
            int si = -1;
            for (size_t k = 0; k < S->streams.size(); ++k)
                if (!S->stream_busy[k]) { si = static_cast<int>(k); break; }
            if (si < 0 || S->queue.empty()) return;
            int admitted_total = 0;
            for (const Launch& x : S->inflight) admitted_total += static_cast<int>(x.jobs.size());
            for (auto it = S->queue.begin(); it != S->queue.end() &&
                                             static_cast<int>(Lh.jobs.size()) < std::min(kMaxPerLaunch, p.requests_per_launch) &&
                                             admitted_total + static_cast<int>(Lh.jobs.size()) < p.max_inflight;) {
                Job& j = *it;
                const std::pair<int, int> kk(j.req.run, j.req.site);
                auto kit = S->key_of.find(kk);
                if (kit != S->key_of.end() && S->key_busy[kit->second]) { ++it; continue; }  // key in flight
                size_t off = 0;
                const size_t need = job_bytes(p, S->nb, L_of(j.req));
                if (!S->arena.alloc(need, &off)) break;       // memory full: keep arrival order
                int key;
                if (kit != S->key_of.end()) {
                    key = kit->second;
                    // fields kept at another L are not a state of this request's chains:
                    // such a request starts cold (and its fields then replace the record's)
                    j.warm = S->key_valid[key] != 0 && S->key_L[key] == j.req.L;
                } else {
                    // new key: a free record, else the least recently used idle one
                    key = -1;
                    if (static_cast<int>(S->key_of.size()) < p.max_keys) {
                        key = static_cast<int>(S->key_of.size());
                    } else {
                        uint64_t best = UINT64_MAX;
                        for (auto& kv : S->key_of)
                            if (!S->key_busy[kv.second] && S->key_used[kv.second] < best) {
                                best = S->key_used[kv.second];
                                key = kv.second;
                            }
                        if (key >= 0) {
                            for (auto e2 = S->key_of.begin(); e2 != S->key_of.end(); ++e2)
                                if (e2->second == key) { S->key_of.erase(e2); break; }
                        }
                    }
                    if (key < 0) { S->arena.release(off, need); break; }
                    S->key_of[kk] = key;
                    S->key_valid[key] = 0;
                    j.warm = false;
                }
                S->key_busy[key] = 1;
                S->key_used[key] = ++S->lru_clock;
                j.key = key;
                j.off = off;
                j.bytes = need;
                Lh.jobs.push_back(j);
                it = S->queue.erase(it);
            }
            if (Lh.jobs.empty()) return;
            Lh.stream = si;
            S->stream_busy[si] = true;
            S->peak_bytes = std::max(S->peak_bytes, S->arena.used());
        }
        cudaEventCreateWithFlags(&Lh.done, cudaEventDisableTiming);
        const hf_status st = start_launch(S, Lh);
        if (st != HF_OK) {
            // fail the jobs of this launch, free their memory
            std::lock_guard<std::mutex> g(S->mu);
            for (const Job& j : Lh.jobs) {
                S->arena.release(j.off, j.bytes);
                S->key_busy[j.key] = 0;
                S->key_valid[j.key] = 0;
                hf_result r{};
                r.ticket = j.ticket;
                r.status = st;
                S->done[j.ticket] = r;
            }
            S->stream_busy[Lh.stream] = false;
            cudaEventDestroy(Lh.done);
            S->cv.notify_all();
            return;
        }
        int n_in = 0;
        S->inflight.push_back(Lh);
        for (const Launch& x : S->inflight) n_in += static_cast<int>(x.jobs.size());
        S->peak_inflight = std::max(S->peak_inflight, n_in);
    }
}

void worker_loop(hf_srv* S) {
    cudaSetDevice(S->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty() && S->inflight.empty()) break;
            if (S->inflight.empty() && S->queue.empty())
                S->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
        progress(S);
        if (!S->inflight.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

hf_status hf_srv_workspace_size(const hf_srv_params* p, size_t* bytes) {
    std::string e;
    if (validate_srv(p, e) != HF_OK) return sfail(nullptr, HF_EINVAL, e);
    if (!bytes) return sfail(nullptr, HF_EINVAL, "null bytes pointer");
    const int nb = p->n_measure / p->bin_size;
    // the warm-start store plus room for max_inflight requests at the largest L
    *bytes = warm_bytes(*p) + static_cast<size_t>(p->max_inflight) * job_bytes(*p, nb, p->max_L) + 256;
    return HF_OK;
}

hf_status hf_srv_create(const hf_srv_params* p, void* d_pool, size_t pool_bytes, hf_srv** out) {
    if (!out) return sfail(nullptr, HF_EINVAL, "null output handle");
    *out = nullptr;
    std::string e;
    if (validate_srv(p, e) != HF_OK) return sfail(nullptr, HF_EINVAL, e);
    if (!d_pool || (reinterpret_cast<uintptr_t>(d_pool) & 255u))
        return sfail(nullptr, HF_EINVAL, "device pool must be non-null and 256-byte aligned");
    const int nb = p->n_measure / p->bin_size;
    const size_t wb = warm_bytes(*p);
    if (pool_bytes < wb + job_bytes(*p, nb, p->max_L))
        return sfail(nullptr, HF_ENOMEM, "device pool too small for the warm-start store and one request");
    hf_srv* S = new (std::nothrow) hf_srv();
    if (!S) return sfail(nullptr, HF_ENOMEM, "host allocation failed");
    S->p = *p;
    if (S->p.requests_per_launch <= 0 || S->p.requests_per_launch > kMaxPerLaunch) S->p.requests_per_launch = kMaxPerLaunch;
    S->nb = nb;
    S->pool = static_cast<char*>(d_pool);
    S->pool_bytes = pool_bytes;
    S->warm_s = reinterpret_cast<int8_t*>(S->pool);
    S->warm_nsw = reinterpret_cast<uint32_t*>(S->pool + align256(static_cast<size_t>(p->chains_per_request) * p->max_L * p->max_keys));
    S->arena_off = wb;
    S->arena.reset(pool_bytes - wb);
    S->key_busy.assign(p->max_keys, 0);
    S->key_valid.assign(p->max_keys, 0);
    S->key_L.assign(p->max_keys, 0);
    S->key_used.assign(p->max_keys, 0);
    cudaError_t ce = cudaGetDevice(&S->device);
    const int ns = p->n_streams;
    S->streams.assign(ns, nullptr);
    S->stream_busy.assign(ns, false);
    for (int k = 0; k < ns && ce == cudaSuccess; ++k) ce = cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking);
    const size_t nin = static_cast<size_t>(ns) * kMaxPerLaunch * 2 * kMaxLServe;
    const size_t nout = static_cast<size_t>(ns) * kMaxPerLaunch * 2 * (2 * kMaxLServe + 4);
    if (ce == cudaSuccess) ce = cudaHostAlloc(&S->h_in, sizeof(double) * nin, cudaHostAllocDefault);
    if (ce == cudaSuccess) ce = cudaHostAlloc(&S->h_out, sizeof(double) * nout, cudaHostAllocDefault);
    if (ce == cudaSuccess) ce = cudaHostAlloc(&S->h_cnt, sizeof(uint32_t) * 2 * ns * kMaxPerLaunch, cudaHostAllocDefault);
    if (ce != cudaSuccess) {
        std::string m = std::string("hf_srv_create: ") + cudaGetErrorString(ce);
        (void)cudaGetLastError();
        hf_srv_free(S);
        return sfail(nullptr, HF_ECUDA, m);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return HF_OK;
}

hf_status hf_srv_submit(hf_srv* S, const hf_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket) return sfail(S, HF_EINVAL, "hf_srv_submit: null argument");
    if (!hfk::qmc_f64_supported(r->L) || r->L > S->p.max_L)
        return sfail(S, HF_EINVAL, "hf_srv_submit: L must be a supported slice count <= max_L");
    if (!(r->beta > 0.0) || !(r->U >= 0.0)) return sfail(S, HF_EINVAL, "hf_srv_submit: need beta > 0, U >= 0");
    for (int sp = 0; sp < 2; ++sp)
        for (int m = 0; m < r->L; ++m)
            if (!std::isfinite(r->g0_tau[sp][m])) return sfail(S, HF_EINVAL, "hf_srv_submit: non-finite bath");
    Job j;
    j.req = *r;
    j.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return sfail(S, HF_EBUSY, "hf_srv_submit: service is shutting down");
        j.ticket = S->next_ticket++;
        S->queue.push_back(j);
    }
    S->cv.notify_all();
    *ticket = j.ticket;
    return HF_OK;
}

hf_status hf_srv_poll(hf_srv* S, uint64_t ticket, hf_result* out) {
    if (!S || !out) return sfail(S, HF_EINVAL, "hf_srv_poll: null argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (ticket == 0 || ticket >= S->next_ticket) return sfail(S, HF_EINVAL, "hf_srv_poll: unknown ticket");
        return HF_ENOTREADY;
    }
    *out = it->second;
    S->done.erase(it);
    return out->status == HF_OK ? HF_OK : static_cast<hf_status>(out->status);
}

hf_status hf_srv_wait(hf_srv* S, uint64_t ticket, double timeout_s, hf_result* out) {
    if (!S || !out) return sfail(S, HF_EINVAL, "hf_srv_wait: null argument");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        auto it = S->done.find(ticket);
        if (it != S->done.end()) {
            *out = it->second;
            S->done.erase(it);
            return out->status == HF_OK ? HF_OK : static_cast<hf_status>(out->status);
        }
        if (ticket == 0 || ticket >= S->next_ticket) return sfail(S, HF_EINVAL, "hf_srv_wait: unknown ticket");
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (S->done.count(ticket)) continue;
            S->err = "hf_srv_wait: timed out";
            return HF_ETIMEOUT;
        }
    }
}

hf_status hf_srv_stats(hf_srv* S, hf_srv_stats_t* out) {
    if (!S || !out) return sfail(S, HF_EINVAL, "hf_srv_stats: null argument");
    std::lock_guard<std::mutex> g(S->mu);
    out->queued = static_cast<int>(S->queue.size());
    int n = 0;
    for (const Launch& x : S->inflight) n += static_cast<int>(x.jobs.size());
    out->inflight = n;
    out->peak_inflight = S->peak_inflight;
    out->completed = S->n_completed;
    out->bytes_in_use = S->arena.used();
    out->peak_bytes = S->peak_bytes;
    out->arena_bytes = S->pool_bytes - S->arena_off;
    out->warm_keys = static_cast<int>(S->key_of.size());
    return HF_OK;
}

void hf_srv_free(hf_srv* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->queue.clear();      // queued work is dropped; admitted launches finish first
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Launch& x : S->inflight) if (x.done) cudaEventDestroy(x.done);
    for (cudaStream_t st : S->streams)
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    if (S->h_in) cudaFreeHost(S->h_in);
    if (S->h_out) cudaFreeHost(S->h_out);
    if (S->h_cnt) cudaFreeHost(S->h_cnt);
    delete S;
}

const char* hf_srv_last_error(const hf_srv* S) { return S ? S->err.c_str() : g_srv_error.c_str(); }

}  // extern "C"
