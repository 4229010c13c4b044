// Serving engine (include/polymul.h, pm_server_*): a request loop that
// batches incoming products continuously.
//
// Requests are admitted in arrival order when a stream slot and enough of
// the engine's device arena (the HBM budget) and pinned staging are free.
// Admitted products that fit the batch kernels are grouped into a batch and
// enqueued with pm_batch_enqueue's workspace mode on one of several streams,
// so batches that arrive while others run overlap on the device; larger
// products go to a worker thread that runs pm_polymul on its own stream.
// Completion is observed with events (no blocking waits on the caller's
// thread); results land directly in the requests' device buffers.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "pm_common.cuh"

namespace pm {
void batch_ws_sizes(const pm_batch_item *items, u32 count, const pm_batch_options *opt, u64 *dbytes, u64 *hbytes);
}

namespace {

using pm::u64;
using pm::u32;

// first-fit allocator over [0, size) with coalescing frees
class Arena {
  public:
    void init(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
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

struct Req {
    pm_batch_item item;
    uint64_t tag;
    double t_submit, t_admit;
};

struct Flight {
    std::vector<Req> reqs;
    std::vector<pm_batch_item> items;
    cudaEvent_t ev;
    size_t doff, dbytes, hoff, hbytes;
    int stream;
};

}  // namespace

struct pm_server {
    pm_server_config cfg;
    int device = 0;
    unsigned char *dbase = nullptr;
    unsigned char *hbase = nullptr;
    Arena darena, harena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::deque<Req> pending;
    std::vector<Flight> flights;
    std::vector<pm_server_done> done;
    std::chrono::steady_clock::time_point t0;
    // worker for products above the batch limits
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> big;
    std::vector<pm_server_done> big_done;
    bool stop = false;
    u32 big_active = 0;
    u32 max_flights_seen = 0;
    u64 launched_batches = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

bool fits_batch(const pm_batch_item &it)
{
    return it.f.n <= PM_BATCH_MAX_TERMS && it.g.n <= PM_BATCH_MAX_TERMS;
}

void worker_loop(pm_server *s)
{
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Req r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->big.empty(); });
            if (s->stop && s->big.empty()) break;
            r = s->big.front();
            s->big.pop_front();
            s->big_active = 1;
        }
        r.t_admit = s->now();
        pm_terms_out h = r.item.h;
        const int rc = pm_polymul(&r.item.pk, r.item.coef_kind, &r.item.f, &r.item.g, &h, nullptr, nullptr, st);
        cudaStreamSynchronize(st);
        pm_server_done d;
        memset(&d, 0, sizeof(d));
        d.tag = r.tag;
        d.status = rc;
        d.n = h.n;
        d.t_submit = r.t_submit;
        d.t_admit = r.t_admit;
        d.t_done = s->now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->big_done.push_back(d);
            s->big_active = 0;
        }
    }
    cudaStreamDestroy(st);
}

void reap(pm_server *s)
{
    for (size_t k = 0; k < s->flights.size();) {
        Flight &f = s->flights[k];
        const cudaError_t e = cudaEventQuery(f.ev);
        if (e == cudaErrorNotReady) {
            k++;
            continue;
        }
        const double t = s->now();
        const int rc = e == cudaSuccess ? PM_OK : PM_ECUDA;
        if (rc == PM_OK) pm_batch_collect(f.items.data(), (u32)f.items.size(), s->hbase + f.hoff);
        for (size_t q = 0; q < f.reqs.size(); q++) {
            pm_server_done d;
            memset(&d, 0, sizeof(d));
            d.tag = f.reqs[q].tag;
            d.status = rc == PM_OK ? f.items[q].status : rc;
            d.n = rc == PM_OK ? f.items[q].h.n : 0;
            d.t_submit = f.reqs[q].t_submit;
            d.t_admit = f.reqs[q].t_admit;
            d.t_done = t;
            s->done.push_back(d);
        }
        cudaEventDestroy(f.ev);
        s->darena.release(f.doff, f.dbytes);
        s->harena.release(f.hoff, f.hbytes);
        s->stream_busy[f.stream] = false;
        s->flights.erase(s->flights.begin() + k);
    }
}

void fail_now(pm_server *s, const Req &r, int code)
{
    pm_server_done d;
    memset(&d, 0, sizeof(d));
    d.tag = r.tag;
    d.status = code;
    d.t_submit = r.t_submit;
    d.t_admit = d.t_done = s->now();
    s->done.push_back(d);
}

// admit and launch as many batches as stream slots and memory allow (the
// pending queue holds only products the batch kernels take)
void launch(pm_server *s)
{
    for (;;) {
        if (s->pending.empty()) return;
        int slot = -1;
        for (size_t k = 0; k < s->streams.size(); k++)
            if (!s->stream_busy[k]) {
                slot = (int)k;
                break;
            }
        if (slot < 0) return;
        // the longest prefix of the queue whose workspace fits
        std::vector<pm_batch_item> items;
        size_t take = 0;
        u64 dbytes = 0, hbytes = 0;
        while (take < s->pending.size() && take < s->cfg.max_batch) {
            items.push_back(s->pending[take].item);
            u64 db = 0, hb = 0;
            try {
                pm::batch_ws_sizes(items.data(), (u32)items.size(), &s->cfg.batch, &db, &hb);
            } catch (const pm::Error &e) {
                items.pop_back();
                if (take == 0) {  // this request is invalid on its own
                    fail_now(s, s->pending.front(), e.code);
                    s->pending.pop_front();
                    goto next_round;
                }
                break;
            }
            if (db > s->cfg.device_budget || hb > s->cfg.host_budget) {
                items.pop_back();
                if (take == 0) {  // can never fit the budget
                    fail_now(s, s->pending.front(), PM_ENOMEM);
                    s->pending.pop_front();
                    goto next_round;
                }
                break;
            }
            dbytes = db;
            hbytes = hb;
            take++;
        }
        if (take == 0) return;
        {
            size_t doff = 0, hoff = 0;
            // shrink the batch until its workspace fits the free memory
            while (take > 0) {
                if (s->darena.alloc(dbytes, doff)) {
                    if (s->harena.alloc(hbytes, hoff)) break;
                    s->darena.release(doff, dbytes);
                }
                take--;
                items.pop_back();
                if (take == 0) break;
                u64 db = 0, hb = 0;
                pm::batch_ws_sizes(items.data(), (u32)items.size(), &s->cfg.batch, &db, &hb);
                dbytes = db;
                hbytes = hb;
            }
            if (take == 0) return;  // wait for memory to free up
            Flight f;
            f.items = items;
            f.doff = doff;
            f.dbytes = dbytes;
            f.hoff = hoff;
            f.hbytes = hbytes;
            f.stream = slot;
            const double t = s->now();
            for (size_t q = 0; q < take; q++) {
                Req r = s->pending.front();
                s->pending.pop_front();
                r.t_admit = t;
                f.reqs.push_back(r);
            }
            const int rc = pm_batch_enqueue(f.items.data(), (u32)take, &s->cfg.batch, s->dbase + doff, dbytes,
                                            s->hbase + hoff, hbytes, s->streams[slot]);
            if (rc != PM_OK) {
                for (auto &r : f.reqs) fail_now(s, r, rc);
                s->darena.release(doff, dbytes);
                s->harena.release(hoff, hbytes);
                continue;
            }
            cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
            cudaEventRecord(f.ev, s->streams[slot]);
            s->stream_busy[slot] = true;
            s->flights.push_back(std::move(f));
            s->launched_batches++;
            if (s->flights.size() > s->max_flights_seen) s->max_flights_seen = (u32)s->flights.size();
        }
    next_round:;
    }
}

}  // namespace

extern "C" int pm_server_create(const pm_server_config *cfg, pm_server **srv)
{
    if (!cfg || !srv) return PM_EINVAL;
    *srv = nullptr;
    pm_server *s = new (std::nothrow) pm_server();
    if (!s) return PM_ENOMEM;
    s->cfg = *cfg;
    if (!s->cfg.device_budget) s->cfg.device_budget = 8ull << 30;
    if (!s->cfg.host_budget) s->cfg.host_budget = 64ull << 20;
    if (!s->cfg.streams) s->cfg.streams = 4;
    if (!s->cfg.max_batch) s->cfg.max_batch = 256;
    if (s->cfg.streams > 64) s->cfg.streams = 64;
    cudaGetDevice(&s->device);
    if (cudaMalloc(&s->dbase, s->cfg.device_budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return PM_ENOMEM;
    }
    if (cudaMallocHost(&s->hbase, s->cfg.host_budget) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->dbase);
        delete s;
        return PM_ENOMEM;
    }
    s->darena.init(s->cfg.device_budget);
    s->harena.init(s->cfg.host_budget);
    for (u32 k = 0; k < s->cfg.streams; k++) {
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        s->streams.push_back(st);
        s->stream_busy.push_back(false);
    }
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(worker_loop, s);
    *srv = s;
    return PM_OK;
}

extern "C" int pm_server_submit(pm_server *s, const pm_batch_item *item, uint64_t tag)
{
    if (!s || !item) return PM_EINVAL;
    Req r;
    r.item = *item;
    r.item.status = 0;
    r.tag = tag;
    r.t_submit = s->now();
    r.t_admit = 0;
    if (fits_batch(r.item)) {
        s->pending.push_back(r);
    } else {
        // too large for the batch kernels: straight to the worker, so it
        // neither waits behind nor splits the batches of small requests
        std::lock_guard<std::mutex> lk(s->mu);
        s->big.push_back(r);
        s->cv.notify_one();
    }
    return PM_OK;
}

extern "C" int pm_server_cancel(pm_server *s, uint64_t tag)
{
    if (!s) return PM_EINVAL;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
        if (it->tag == tag) {
            const Req r = *it;
            s->pending.erase(it);
            fail_now(s, r, PM_ECANCELED);
            return PM_OK;
        }
    Req r;
    bool found = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->big.begin(); it != s->big.end(); ++it)
            if (it->tag == tag) {
                r = *it;
                s->big.erase(it);
                found = true;
                break;
            }
    }
    if (!found) return PM_EINVAL;  // unknown, already admitted, or done
    fail_now(s, r, PM_ECANCELED);
    return PM_OK;
}

extern "C" int pm_server_progress(pm_server *s, pm_server_done *out, uint32_t cap, uint32_t *n_done)
{
    if (!s || !n_done || (cap && !out)) return PM_EINVAL;
    reap(s);
    launch(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &d : s->big_done) s->done.push_back(d);
        s->big_done.clear();
    }
    const uint32_t n = (uint32_t)(s->done.size() < cap ? s->done.size() : cap);
    for (uint32_t k = 0; k < n; k++) out[k] = s->done[k];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_done = n;
    return PM_OK;
}

extern "C" int pm_server_state(pm_server *s, pm_server_state_t *st)
{
    if (!s || !st) return PM_EINVAL;
    memset(st, 0, sizeof(*st));
    st->queued = (uint32_t)s->pending.size();
    st->in_flight = (uint32_t)s->flights.size();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        st->big_queued = (uint32_t)s->big.size();
        st->big_active = s->big_active;
    }
    st->max_in_flight = s->max_flights_seen;
    st->batches = s->launched_batches;
    st->device_used = s->darena.used();
    st->clock = s->now();
    return PM_OK;
}

extern "C" void pm_server_destroy(pm_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &f : s->flights) {
        cudaEventSynchronize(f.ev);
        cudaEventDestroy(f.ev);
    }
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    cudaFree(s->dbase);
    cudaFreeHost(s->hbase);
    delete s;
}
