// Serving loop (a10): continuous batching of alignment requests.  Not in
// the paper (its Sec. 3.2 distributes a fixed set of pairs over MPI ranks;
// here requests keep arriving and share one GPU).
//
// Requests wait in a FIFO.  Each of W worker threads owns a context (its
// own CUDA stream, scratch pool and error word) and repeatedly admits the
// oldest requests into a batch while (a) the batch has room and (b) the
// traceback buffers the whole server has in flight stay within the budget
// -- a CIGAR request reserves the pointer bytes of its full grid,
// ceil((m+1)(n+1)/4) rounded up to 256, the most its alignment can need if
// the band falls back; a score-only request reserves nothing.  The worker
// runs the batch through the batched path (certified learned band with
// fallback when the server was created with NW_LEARNED_BAND), whose work
// queue is device-resident (task array + atomic head), then publishes the
// results and releases its reservation.  Batches of different workers run
// on different streams, so requests that arrive while others are on the
// GPU are admitted as soon as a worker and memory are free, and their
// kernels overlap on the device.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "nw_internal.cuh"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket;
    std::vector<uint8_t> a2b, b2b;
    uint32_t m, n;
    bool cigar;
    double t_submit;
    uint64_t reserve;
};

struct Done {
    uint64_t ticket;
    int32_t status, score;
    std::string cigar;
    double latency;
};

}  // namespace

struct nw_server {
    int device = 0;
    nw_scoring sc{};
    uint32_t flags = 0;
    uint64_t budget = 0;
    uint32_t max_batch = 0;
    std::vector<nw_ctx *> ctxs;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::deque<Done> done;
    uint64_t reserved = 0, inflight = 0;
    uint64_t submitted = 0, completed = 0, cells_done = 0, batches = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::string msg;
};

static uint64_t trace_reserve(uint32_t m, uint32_t n, bool cigar) {
    if (!cigar) return 0;
    const uint64_t b = ((uint64_t)m + 1) * ((uint64_t)n + 1);
    return (((b + 3) / 4) + 255) / 256 * 256;
}

static void worker_loop(nw_server *srv, nw_ctx *ctx) {
    cudaSetDevice(srv->device);
    std::vector<uint8_t> pool;
    std::vector<uint64_t> ao, bo, coff;
    std::vector<uint32_t> al, bl;
    std::vector<int32_t> scores;
    std::vector<uint64_t> clen;
    std::vector<char> cig;
    for (;;) {
        std::vector<Req> batch;
        uint64_t res = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || !srv->pending.empty(); });
            if (srv->stop && srv->pending.empty()) return;
            while (!srv->pending.empty() && batch.size() < srv->max_batch) {
                const Req &r = srv->pending.front();
                // admit while the traceback buffers in flight fit the budget;
                // a request alone on an idle server is always admitted
                if (srv->reserved + res + r.reserve > srv->budget && !(srv->reserved + res == 0)) break;
                res += r.reserve;
                batch.push_back(std::move(srv->pending.front()));
                srv->pending.pop_front();
            }
            srv->reserved += res;
            srv->inflight += batch.size();
        }
        if (batch.empty()) continue;
        std::vector<Done> out(batch.size());
        uint64_t cells = 0;
        // two sub-batches: score-only requests, then CIGAR requests
        for (int want = 0; want < 2; ++want) {
            std::vector<size_t> idx;
            for (size_t k = 0; k < batch.size(); ++k)
                if ((int)batch[k].cigar == want) idx.push_back(k);
            if (idx.empty()) continue;
            pool.clear();
            ao.clear();
            bo.clear();
            al.clear();
            bl.clear();
            coff.assign(1, 0);
            for (size_t k : idx) {
                const Req &r = batch[k];
                auto add = [&](const std::vector<uint8_t> &s) {
                    const uint64_t off = pool.size();
                    pool.insert(pool.end(), s.begin(), s.end());
                    pool.resize((pool.size() + 15) / 16 * 16, 0);
                    return off;
                };
                ao.push_back(add(r.a2b));
                bo.push_back(add(r.b2b));
                al.push_back(r.m);
                bl.push_back(r.n);
                coff.push_back(coff.back() + (want ? nw_cigar_bound(r.m, r.n) : 0));
                cells += (uint64_t)r.m * r.n;
            }
            if (pool.empty()) pool.resize(16, 0);
            const uint32_t np = (uint32_t)idx.size();
            scores.assign(np, 0);
            clen.assign(np, 0);
            cig.assign(want ? coff.back() + 1 : 1, 0);
            const uint32_t fl = (want ? NW_CIGAR : 0u) | NW_HOST_IO | (srv->flags & (NW_LEARNED_BAND | NW_CIGAR_M));
            const int rc = nw_align_batch(ctx, pool.data(), ao.data(), al.data(), bo.data(), bl.data(), np, srv->sc, fl,
                                          scores.data(), want ? cig.data() : nullptr, want ? coff.data() : nullptr,
                                          want ? clen.data() : nullptr);
            for (uint32_t q = 0; q < np; ++q) {
                Done &d = out[idx[q]];
                d.ticket = batch[idx[q]].ticket;
                d.status = rc;
                d.score = rc == NW_OK ? scores[q] : 0;
                if (want && rc == NW_OK) d.cigar.assign(cig.data() + coff[q], clen[q]);
            }
        }
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (size_t k = 0; k < batch.size(); ++k) {
                out[k].latency = t - batch[k].t_submit;
                srv->done.push_back(std::move(out[k]));
            }
            srv->reserved -= res;
            srv->inflight -= batch.size();
            srv->completed += batch.size();
            srv->cells_done += cells;
            srv->batches += 1;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
}

using namespace nw;

extern "C" {

nw_server *nw_server_create(nw_ctx *ctx, uint32_t workers, uint32_t max_batch, uint64_t trace_budget, nw_scoring sc,
                            uint32_t flags) {
    if (!ctx || workers == 0 || workers > 16 || max_batch == 0) return nullptr;
    if (check_scoring(ctx, sc) != NW_OK) return nullptr;
    nw_server *srv = new nw_server();
    srv->device = ctx->device;
    srv->sc = sc;
    srv->flags = flags;
    srv->budget = trace_budget;
    srv->max_batch = max_batch;
    // every worker gets its own context and stream; the learned model (if
    // the parent has one) is copied into each
    std::vector<float> params;
    if (ctx->band_model) {
        params.resize(nw_band_model_size());
        if (nw_band_model_get(ctx, params.data(), params.size()) != NW_OK) params.clear();
    }
    const uint64_t per = ctx->budget / (workers + 1);
    for (uint32_t w = 0; w < workers; ++w) {
        cudaSetDevice(ctx->device);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            nw_server_destroy(srv);
            return nullptr;
        }
        nw_ctx *c = nw_ctx_create(ctx->device, st, per);
        if (!c) {
            cudaStreamDestroy(st);
            nw_server_destroy(srv);
            return nullptr;
        }
        if (!params.empty()) nw_band_model_set(c, params.data(), params.size());
        srv->ctxs.push_back(c);
    }
    for (nw_ctx *c : srv->ctxs) srv->workers.emplace_back(worker_loop, srv, c);
    return srv;
}

int nw_server_submit(nw_server *srv, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                     uint32_t want_cigar, uint64_t *ticket) {
    if (!srv || (m && !a2b) || (n && !b2b)) return NW_ERR_ARG;
    if (m >= (1u << 30) || n >= (1u << 30)) return NW_ERR_ARG;
    Req r;
    r.a2b.assign(a2b, a2b + (m + 3) / 4);
    r.b2b.assign(b2b, b2b + (n + 3) / 4);
    r.m = m;
    r.n = n;
    r.cigar = want_cigar != 0;
    r.reserve = trace_reserve(m, n, r.cigar);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return NW_ERR_ARG;
        r.ticket = srv->next_ticket++;
        r.t_submit = now_s();
        if (ticket) *ticket = r.ticket;
        srv->pending.push_back(std::move(r));
        srv->submitted += 1;
    }
    srv->cv_work.notify_one();
    return NW_OK;
}

int nw_server_submit_many(nw_server *srv, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                          const uint64_t *b_off, const uint32_t *b_len, const uint8_t *want_cigar, uint32_t count,
                          uint64_t *tickets) {
    if (!srv || (count && (!pool2b || !a_off || !a_len || !b_off || !b_len || !want_cigar))) return NW_ERR_ARG;
    std::vector<Req> reqs(count);
    for (uint32_t k = 0; k < count; ++k) {
        if (a_len[k] >= (1u << 30) || b_len[k] >= (1u << 30)) return NW_ERR_ARG;
        Req &r = reqs[k];
        r.a2b.assign(pool2b + a_off[k], pool2b + a_off[k] + (a_len[k] + 3) / 4);
        r.b2b.assign(pool2b + b_off[k], pool2b + b_off[k] + (b_len[k] + 3) / 4);
        r.m = a_len[k];
        r.n = b_len[k];
        r.cigar = want_cigar[k] != 0;
        r.reserve = trace_reserve(r.m, r.n, r.cigar);
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return NW_ERR_ARG;
        const double t = now_s();
        for (uint32_t k = 0; k < count; ++k) {
            reqs[k].ticket = srv->next_ticket++;
            reqs[k].t_submit = t;
            if (tickets) tickets[k] = reqs[k].ticket;
            srv->pending.push_back(std::move(reqs[k]));
        }
        srv->submitted += count;
    }
    srv->cv_work.notify_all();
    return NW_OK;
}

int nw_server_poll(nw_server *srv, nw_completion *out, uint32_t cap, uint32_t *count, char *cigar_buf,
                   uint64_t cigar_cap, uint64_t *cigar_used) {
    if (!srv || !count || (cap && !out)) return NW_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    uint32_t k = 0;
    uint64_t used = 0;
    while (k < cap && !srv->done.empty()) {
        Done &d = srv->done.front();
        const uint64_t need = d.cigar.empty() ? 0 : d.cigar.size() + 1;
        if (need && (!cigar_buf || used + need > cigar_cap)) {
            if (k == 0) {  // the oldest CIGAR alone does not fit: report its size, move nothing
                *count = 0;
                if (cigar_used) *cigar_used = need;
                return NW_ERR_CIGAR_TRUNC;
            }
            break;
        }
        out[k].ticket = d.ticket;
        out[k].status = d.status;
        out[k].score = d.score;
        out[k].cigar_len = d.cigar.size();
        out[k].cigar_off = need ? used : 0;
        out[k].latency_s = d.latency;
        if (need) {
            memcpy(cigar_buf + used, d.cigar.c_str(), need);
            used += need;
        }
        srv->done.pop_front();
        ++k;
    }
    *count = k;
    if (cigar_used) *cigar_used = used;
    return NW_OK;
}

int nw_server_drain(nw_server *srv, double timeout_s) {
    if (!srv) return NW_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                          [&] { return srv->pending.empty() && srv->inflight == 0; });
    return ok ? NW_OK : NW_ERR_TIMEOUT;
}

int nw_server_stats(nw_server *srv, uint64_t *out, int cap) {
    if (!srv || !out) return -NW_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t v[8] = {srv->submitted, srv->completed, (uint64_t)srv->pending.size(), srv->inflight,
                           srv->cells_done, srv->reserved, srv->batches, srv->budget};
    for (int k = 0; k < cap && k < 8; ++k) out[k] = v[k];
    return 8;
}

void nw_server_destroy(nw_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers)
        if (t.joinable()) t.join();
    for (nw_ctx *c : srv->ctxs) {
        cudaStream_t st = c->stream;
        nw_ctx_destroy(c);
        if (st) cudaStreamDestroy(st);
    }
    delete srv;
}

}  // extern "C"
