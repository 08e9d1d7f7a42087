// Serving loop of the KLB library (declared in include/klb.h): a first come,
// first served admission queue over a caller-provided device arena, lattices
// resident until their residual converges, and one batch re-formed whenever
// the resident set changes.  Built on the public lattice and batch calls.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "klb.h"
#include "klb_internal.h"

namespace {

thread_local std::string g_server_error;

constexpr size_t kAlign = 256;

size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over byte offsets [0, size) in 256-byte units.  Free
// blocks are keyed by offset; a released block merges with free neighbours.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        size_ = size / kAlign * kAlign;
        if (size_) free_[0] = size_;
        used_ = peak_ = 0;
    }

    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, next = it->first + bytes;
            free_.erase(it);
            if (rest) free_[next] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }

    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        size_t start = off, len = bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + bytes == next->first) {
            len += next->second;
            free_.erase(next);
        }
        free_[start] = len;
        used_ -= bytes;
    }

    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
    klb_request r;
    std::vector<uint8_t> mask;  // MASK cross-section, owned copy
    size_t bytes = 0;
    int64_t sites = 0;
};

struct Resident {
    Request q;
    klb_lattice *L = nullptr;
    size_t off = 0;
    double admitted = 0;
};

}  // namespace

struct klb_server {
    char *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t stream = nullptr;
    klb_server_opts o{};
    size_t table_bytes = 0;  // reserved at the start of the arena
    Arena heap;              // lattices, after the table region
    std::deque<Request> queue;
    std::vector<Resident> res;
    klb_batch *batch = nullptr;
    bool reform = false;
    std::deque<klb_result> done;
    double *host_sums = nullptr;  // pinned, max_resident x kNumSums (retirement checks)
    klb_server_stats stats{};
    std::chrono::steady_clock::time_point t0;
    std::string err;
};

namespace {

klb_status sfail(klb_server *S, klb_status st, const std::string &msg)
{
    if (S)
        S->err = msg;
    else
        g_server_error = msg;
    return st;
}

double now(const klb_server *S)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

void drop_batch(klb_server *S)
{
    if (S->batch) klb_batch_destroy(S->batch);
    S->batch = nullptr;
}

void finish(klb_server *S, Resident &r, klb_status status, const klb_obs *obs)
{
    klb_result out;
    std::memset(&out, 0, sizeof out);
    out.id = r.q.r.id;
    out.status = status;
    out.steps = r.L ? klb_get_step(r.L) : 0;
    out.sites = r.q.sites;
    out.bytes = round_up(r.q.bytes);
    out.arrival = r.q.r.arrival;
    out.admitted = r.admitted;
    out.finished = now(S);
    if (obs) out.obs = *obs;
    S->done.push_back(out);
    if (r.L) klb_destroy(r.L);
    r.L = nullptr;
    S->heap.release(r.off, r.q.bytes);
    ++S->stats.finished;
}

// Retirement checks of every resident lattice (waits for the last round).
klb_status retire(klb_server *S)
{
    std::vector<klb_status> verdict(S->res.size(), KLB_OK);
    std::vector<klb_obs> obs(S->res.size());
    std::vector<char> leave(S->res.size(), 0);
    const double t = now(S);
    // every resident lattice runs on the server's stream: enqueue all
    // observation passes, synchronise once
    if (!S->host_sums && !S->res.empty()) {
        const size_t bytes = sizeof(double) * klb::kNumSums * (size_t)S->o.max_resident;
        if (cudaMallocHost((void **)&S->host_sums, bytes) != cudaSuccess) {
            S->host_sums = nullptr;
            return sfail(S, KLB_ECUDA, "pinned host memory for the retirement checks");
        }
    }
    for (size_t k = 0; k < S->res.size(); ++k) {
        const cudaError_t e = klb::observe_enqueue(S->res[k].L, S->host_sums + k * klb::kNumSums);
        if (e != cudaSuccess) return sfail(S, KLB_ECUDA, std::string("observation: ") + cudaGetErrorString(e));
    }
    if (!S->res.empty()) {
        const cudaError_t e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) return sfail(S, KLB_ECUDA, std::string("observation: ") + cudaGetErrorString(e));
    }
    for (size_t k = 0; k < S->res.size(); ++k) {
        Resident &r = S->res[k];
        const klb_status st = klb::observe_finish(r.L, S->host_sums + k * klb::kNumSums, &obs[k]);
        const int64_t steps = klb_get_step(r.L);
        if (st != KLB_OK) {
            verdict[k] = st;  // KLB_EUNSTABLE
            leave[k] = 1;
        } else if (!std::isnan(obs[k].residual) && obs[k].residual <= r.q.r.tol) {
            leave[k] = 1;
        } else if (steps >= r.q.r.max_steps ||
                   (r.q.r.max_seconds > 0 && t - r.q.r.arrival >= r.q.r.max_seconds)) {
            verdict[k] = KLB_ETIMEOUT;
            leave[k] = 1;
        }
    }
    if (std::find(leave.begin(), leave.end(), 1) == leave.end()) return KLB_OK;
    drop_batch(S);  // holds pointers to the members
    std::vector<Resident> keep;
    for (size_t k = 0; k < S->res.size(); ++k) {
        if (leave[k])
            finish(S, S->res[k], verdict[k], &obs[k]);
        else
            keep.push_back(std::move(S->res[k]));
    }
    S->res.swap(keep);
    S->reform = true;
    return KLB_OK;
}

// Admissions, oldest first, while the oldest fits.
void admit(klb_server *S)
{
    const double t = now(S);
    while (!S->queue.empty() && (int)S->res.size() < S->o.max_resident) {
        Request &q = S->queue.front();
        if (q.r.arrival > t) break;
        size_t off = 0;
        if (!S->heap.alloc(q.bytes, &off)) break;
        Resident r;
        r.q = std::move(q);
        S->queue.pop_front();
        r.off = off;
        r.admitted = t;
        klb_desc d = r.q.r.desc;
        if (d.geom == KLB_GEOM_MASK) d.mask = r.q.mask.data();
        klb_status st = klb_create_lattice(&d, S->arena + S->table_bytes + off, r.q.bytes, S->stream, &r.L);
        if (st == KLB_OK) st = klb_set_couplings(r.L, &r.q.r.couplings);
        if (st != KLB_OK) {
            finish(S, r, st, nullptr);
            continue;
        }
        S->res.push_back(std::move(r));
        S->reform = true;
    }
}

}  // namespace

extern "C" {

size_t klb_server_table_bytes(int storage, int max_resident)
{
    return round_up(klb::batch_table_bytes(storage, max_resident));
}

klb_status klb_server_create(void *arena, size_t arena_bytes, void *stream,
                             const klb_server_opts *opts, klb_server **out)
{
    if (!out || !opts) return sfail(nullptr, KLB_EINVAL, "null argument");
    *out = nullptr;
    const klb_server_opts &o = *opts;
    if (o.kind != KLB_D2Q9 && o.kind != KLB_D3Q19) return sfail(nullptr, KLB_EINVAL, "kind must be KLB_D2Q9 or KLB_D3Q19");
    if (o.storage < KLB_FP64 || o.storage > KLB_BF16_DEV) return sfail(nullptr, KLB_EINVAL, "unknown storage");
    if (o.check_every < 1 || o.max_resident < 1 || o.autotune_steps < 0)
        return sfail(nullptr, KLB_EINVAL, "check_every and max_resident must be >= 1, autotune_steps >= 0");
    if (o.autotune_steps > 0 && (int64_t)o.check_every < 3 * ((int64_t)o.autotune_steps + 1) + 1)
        return sfail(nullptr, KLB_EINVAL, "check_every must exceed 3 (autotune_steps + 1)");
    if (!arena || ((uintptr_t)arena & (kAlign - 1)))
        return sfail(nullptr, KLB_EINVAL, "arena must be a 256-byte aligned device pointer");
    const size_t tb = klb_server_table_bytes(o.storage, o.max_resident);
    if (arena_bytes <= tb) return sfail(nullptr, KLB_ENOMEM, "arena smaller than the batch table region");
    klb_server *S = new (std::nothrow) klb_server();
    if (!S) return sfail(nullptr, KLB_ENOMEM, "host allocation failed");
    S->arena = static_cast<char *>(arena);
    S->arena_bytes = arena_bytes;
    S->stream = static_cast<cudaStream_t>(stream);
    S->o = o;
    S->table_bytes = tb;
    S->heap.reset(arena_bytes - tb);
    S->t0 = std::chrono::steady_clock::now();
    S->stats.arena_bytes = arena_bytes;
    S->stats.table_bytes = tb;
    *out = S;
    return KLB_OK;
}

klb_status klb_server_submit(klb_server *S, const klb_request *req)
{
    if (!S || !req) return sfail(S, KLB_EINVAL, "null argument");
    const klb_request &r = *req;
    if (r.desc.kind != S->o.kind || r.desc.storage != S->o.storage)
        return sfail(S, KLB_EINVAL, "request kind or storage differs from the server's");
    if (!(r.tol > 0) || !std::isfinite(r.tol)) return sfail(S, KLB_EINVAL, "tol must be finite and > 0");
    if (r.max_steps < 1) return sfail(S, KLB_EINVAL, "max_steps must be >= 1");
    if (!(r.max_seconds >= 0) || !std::isfinite(r.max_seconds))
        return sfail(S, KLB_EINVAL, "max_seconds must be finite and >= 0");
    const klb_couplings &c = r.couplings;
    if (!std::isfinite(c.g_we) || !std::isfinite(c.g_wp) || !std::isfinite(c.g_ep) ||
        !std::isfinite(c.g_ec) || !std::isfinite(c.g_pc))
        return sfail(S, KLB_EINVAL, "non-finite coupling");
    klb_info info;
    if (klb_lattice_info(&r.desc, &info) != KLB_OK)
        return sfail(S, KLB_EINVAL, std::string("invalid description: ") + klb_last_error(nullptr));
    if (round_up(info.bytes) > S->heap.size())
        return sfail(S, KLB_EINVAL, "the lattice can never fit in the arena");
    Request q;
    q.r = r;
    q.bytes = info.bytes;
    q.sites = info.active_sites;
    if (r.desc.geom == KLB_GEOM_MASK) {
        q.mask.assign(r.desc.mask, r.desc.mask + (size_t)r.desc.ny * r.desc.nz);
        q.r.desc.mask = nullptr;
    }
    if (q.r.arrival < 0) q.r.arrival = now(S);
    S->queue.push_back(std::move(q));
    return KLB_OK;
}

klb_status klb_server_tick(klb_server *S, int64_t *n_finished)
{
    if (!S) return sfail(S, KLB_EINVAL, "null handle");
    klb_status st = retire(S);
    if (st != KLB_OK) return st;
    admit(S);
    if (S->res.empty()) {
        drop_batch(S);
        S->reform = false;
    } else {
        int64_t steps = S->o.check_every;
        if (S->reform || !S->batch) {
            drop_batch(S);
            std::vector<klb_lattice *> mem;
            for (Resident &r : S->res) mem.push_back(r.L);
            st = klb_batch_create(mem.data(), (int)mem.size(), S->arena, S->table_bytes, &S->batch);
            if (st != KLB_OK) return sfail(S, st, std::string("batch: ") + klb_last_error(nullptr));
            ++S->stats.batch_forms;
            S->reform = false;
            if (S->o.autotune_steps > 0) {
                int w = 0;
                st = klb_batch_autotune(S->batch, S->o.autotune_steps, &w);
                if (st != KLB_OK) return sfail(S, st, std::string("autotune: ") + klb_batch_last_error(S->batch));
                steps -= 3 * ((int64_t)S->o.autotune_steps + 1);
            }
        }
        st = klb_batch_step(S->batch, steps);
        if (st != KLB_OK) return sfail(S, st, std::string("batch step: ") + klb_batch_last_error(S->batch));
        double sites = 0;
        for (const Resident &r : S->res) sites += (double)r.q.sites;
        S->stats.site_updates += sites * S->o.check_every;
        ++S->stats.rounds;
    }
    if (n_finished) *n_finished = (int64_t)S->done.size();
    return KLB_OK;
}

int64_t klb_server_poll(klb_server *S, klb_result *out, int64_t max)
{
    if (!S || !out || max < 1) return 0;
    int64_t n = 0;
    while (n < max && !S->done.empty()) {
        out[n++] = S->done.front();
        S->done.pop_front();
    }
    return n;
}

klb_status klb_server_get_stats(const klb_server *S, klb_server_stats *st)
{
    if (!S || !st) return KLB_EINVAL;
    *st = S->stats;
    st->queued = (int64_t)S->queue.size();
    st->resident = (int64_t)S->res.size();
    st->bytes_in_use = S->heap.used();
    st->peak_bytes_in_use = S->heap.peak();
    st->width = S->batch ? klb_batch_width(S->batch) : 0;
    return KLB_OK;
}

double klb_server_clock(const klb_server *S) { return S ? now(S) : 0.0; }

klb_status klb_server_destroy(klb_server *S)
{
    if (!S) return KLB_OK;
    drop_batch(S);
    for (Resident &r : S->res)
        if (r.L) klb_destroy(r.L);
    if (S->host_sums) cudaFreeHost(S->host_sums);
    delete S;
    return KLB_OK;
}

const char *klb_server_last_error(const klb_server *S) { return S ? S->err.c_str() : g_server_error.c_str(); }

}  // extern "C"
