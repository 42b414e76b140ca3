// Serving loop (a10): continuous batching of alignment requests.  Not in
// the paper (its Sec. 3.2 distributes a fixed set of pairs over MPI ranks;
// here requests keep arriving and share one GPU).
//
// The queue lives on the device.  Submitting a request copies its 2-bit
// sequences into a device arena and its descriptor (arena offsets, lengths,
// traceback reservation, ticket) into a device ring of slots; the host only
// publishes how many requests the ring holds.  The queue's consumer state --
// how many requests have been admitted and how many traceback bytes are
// reserved in flight -- is one 64-bit device word.  Admission and dispatch
// run on the device (k_admit): a warp scans the oldest waiting descriptors,
// admits them in order while the batch has room and the reserved bytes stay
// within the budget (a CIGAR request reserves the pointer bytes of its full
// grid, ceil((m+1)(n+1)/4) rounded up to 256 -- the most its alignment can
// need if the band falls back; a score-only request reserves nothing; a
// request alone on an idle server is always admitted), claims them with one
// compare-and-swap on the queue word, and hands the worker the admitted
// descriptors.  Each of W worker threads owns a context (its own CUDA
// stream, scratch pool and error word); it runs its admitted batch straight
// from the arena through the batched path (certified learned band with
// fallback when the server was created with NW_LEARNED_BAND), whose work
// queue inside the batch is device-resident too (task array + atomic head),
// returns the reservation on the device (k_release), then publishes the
// results.  Batches of different workers run on different streams, so
// requests that arrive while others are on the GPU are admitted as soon as
// a worker and memory are free, and their kernels overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "nw_internal.cuh"

using namespace nw;

namespace {

constexpr uint64_t kUnit = 256;          // reservation granularity (bytes)
constexpr uint32_t kAdmitTries = 1u << 16;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// One slot of the device ring (40 bytes).
struct DevReq {
    uint64_t a_off, b_off;  // byte offsets of the 2-bit sequences in the arena
    uint64_t ticket;
    uint32_t m, n;
    uint32_t units;  // traceback reservation in 256-byte units (0: score only)
    uint32_t cigar;  // 1: the CIGAR is wanted
};

// The consumer side of the queue: high 32 bits = requests admitted so far
// (the ring's head), low 32 bits = reservation units in flight.
struct DevQueue {
    unsigned long long state;
};

// What one admission returns to its worker (followed by the admitted
// descriptors, in queue order).
struct AdmitOut {
    uint32_t head0, count, units, status;
};

// Device admission (one warp).  `tail` is the number of requests published
// when the worker's stream waited for the intake copies; the warp admits a
// prefix of [head, tail) of at most max_batch requests whose reservations
// fit the budget (the first request always fits when nothing is reserved),
// claims it with a compare-and-swap of the queue word, and copies the
// admitted descriptors out.  A lost race with another worker retries from
// the new state (bounded; NW_ERR_TIMEOUT if it never settles).
__global__ void k_admit(DevQueue *q, const DevReq *ring, uint32_t mask, uint32_t tail, uint32_t max_batch,
                        uint32_t budget_units, AdmitOut *out, DevReq *picked, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    for (uint32_t attempt = 0; attempt < kAdmitTries; ++attempt) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(&q->state, 0ull);  // coherent read of the queue word
        s = __shfl_sync(kFull, s, 0);
        const uint32_t head = (uint32_t)(s >> 32), reserved = (uint32_t)s;
        const int32_t waiting = (int32_t)(tail - head);  // <= 0: others took everything published
        const uint32_t lim = waiting > 0 ? min((uint32_t)waiting, max_batch) : 0u;
        uint32_t count = 0;
        uint64_t res = 0;
        for (uint32_t base = 0; base < lim; base += 32) {
            const uint32_t i = base + lane;
            const uint64_t u = i < lim ? ring[(head + i) & mask].units : 0u;
            uint64_t cum = u;  // inclusive prefix sum over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t x = __shfl_up_sync(kFull, cum, d);
                if (lane >= d) cum += x;
            }
            const uint64_t before = (uint64_t)reserved + res + cum - u;  // in flight ahead of request i
            const bool ok = i < lim && (before + u <= budget_units || before == 0);
            const uint32_t bad = __ballot_sync(kFull, !ok);
            const int f = bad ? __ffs(bad) - 1 : 32;  // admitted lanes of this chunk
            count += (uint32_t)f;
            if (f > 0) res += __shfl_sync(kFull, cum, f - 1);
            if (f < 32) break;
        }
        if (count == 0) {
            if (lane == 0) *out = AdmitOut{head, 0u, 0u, 0u};
            return;
        }
        const unsigned long long ns = ((unsigned long long)(head + count) << 32) | (uint32_t)(reserved + res);
        unsigned long long old = 0;
        if (lane == 0) old = atomicCAS(&q->state, s, ns);
        old = __shfl_sync(kFull, old, 0);
        if (old == s) {
            for (uint32_t k = lane; k < count; k += 32) picked[k] = ring[(head + k) & mask];
            if (lane == 0) *out = AdmitOut{head, count, (uint32_t)res, 0u};
            return;
        }
    }
    if (lane == 0) {
        *out = AdmitOut{0u, 0u, 0u, (uint32_t)NW_ERR_TIMEOUT};
        raise_error(err, NW_ERR_TIMEOUT, 0x50000u);
    }
}

// Return a batch's reservation (the queue word's low half never borrows:
// it holds at least the units this batch reserved).
__global__ void k_release(DevQueue *q, uint32_t units) {
    if (threadIdx.x == 0 && units) atomicAdd(&q->state, 0ull - (unsigned long long)units);
}

struct Live {  // a published or staged request, in ticket order
    uint64_t start;  // absolute arena position of its bytes
    double t_submit;
    bool done;
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
    uint32_t budget_units = 0;
    uint32_t max_batch = 0;
    std::vector<nw_ctx *> ctxs;
    std::vector<std::thread> workers;
    // device queue
    uint8_t *arena = nullptr;
    uint64_t arena_bytes = 0;
    DevReq *ring = nullptr;
    uint32_t slots = 0;
    DevQueue *dq = nullptr;
    cudaStream_t intake = nullptr;
    cudaEvent_t intake_ev = nullptr;
    std::mutex intake_mu;  // one submitter at a time (taken before mu)
    // host bookkeeping (mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Live> live;       // requests not yet completed, oldest first
    uint64_t live_front = 0;     // queue index of live.front()
    uint64_t arena_tail = 0;     // next free absolute arena position
    uint64_t tail = 0;           // requests published to the device
    uint64_t head_host = 0;      // requests admitted (sum of the admissions seen)
    uint64_t epoch = 0;          // bumped by every publication and completion
    std::deque<Done> done;
    uint64_t reserved = 0, inflight = 0;
    uint64_t submitted = 0, completed = 0, cells_done = 0, batches = 0;
    bool stop = false;
    // the last batch that failed: its status and its context's message
    uint64_t failed_batches = 0;
    std::string last_error;
};

static uint64_t trace_reserve(uint32_t m, uint32_t n, bool cigar) {
    if (!cigar) return 0;
    const uint64_t b = ((uint64_t)m + 1) * ((uint64_t)n + 1);
    return (((b + 3) / 4) + kUnit - 1) / kUnit * kUnit;
}

static void worker_loop(nw_server *srv, nw_ctx *ctx) {
    cudaSetDevice(srv->device);
    const size_t out_bytes = sizeof(AdmitOut) + (size_t)srv->max_batch * sizeof(DevReq);
    void *d_out = nullptr, *h_out = nullptr;
    if (cudaMalloc(&d_out, out_bytes) != cudaSuccess || cudaMallocHost(&h_out, out_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (d_out) cudaFree(d_out);
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;  // a worker without buffers cannot serve; the others still drain
        return;
    }
    AdmitOut *hdr = (AdmitOut *)h_out;
    const DevReq *picked = (const DevReq *)((char *)h_out + sizeof(AdmitOut));
    std::vector<uint64_t> ao, bo, coff;
    std::vector<uint32_t> al, bl;
    std::vector<int32_t> scores;
    std::vector<uint64_t> clen;
    std::vector<char> cig;
    uint64_t failed_epoch = ~0ull;
    for (;;) {
        uint64_t seen_epoch;
        uint32_t tail_seen;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                return (srv->stop && srv->tail == srv->head_host) ||
                       (srv->tail > srv->head_host && srv->epoch != failed_epoch);
            });
            if (srv->tail == srv->head_host) break;  // stopping, nothing waits
            seen_epoch = srv->epoch;
            tail_seen = (uint32_t)srv->tail;
            // the intake copies of everything published so far come first
            cudaStreamWaitEvent(ctx->stream, srv->intake_ev, 0);
        }
        {
            LaunchTimer t(ctx, "admit");
            k_admit<<<1, 32, 0, ctx->stream>>>(srv->dq, srv->ring, srv->slots - 1, tail_seen, srv->max_batch,
                                               srv->budget_units, (AdmitOut *)d_out,
                                               (DevReq *)((char *)d_out + sizeof(AdmitOut)), ctx->d_err);
        }
        cudaMemcpyAsync(h_out, d_out, out_bytes, cudaMemcpyDeviceToHost, ctx->stream);
        const int arc = nw_ctx_sync(ctx);
        if (arc != NW_OK || hdr->status != 0 || hdr->count == 0) {
            std::lock_guard<std::mutex> lk(srv->mu);
            failed_epoch = seen_epoch;  // wait for a publication or a completion
            continue;
        }
        const uint32_t count = hdr->count, units = hdr->units;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->head_host += count;
            srv->inflight += count;
            srv->reserved += (uint64_t)units * kUnit;
        }
        failed_epoch = ~0ull;
        std::vector<Done> out(count);
        uint64_t cells = 0;
        // two sub-batches: score-only requests, then CIGAR requests; the
        // sequences are read in place from the arena
        for (uint32_t want = 0; want < 2; ++want) {
            std::vector<uint32_t> idx;
            for (uint32_t k = 0; k < count; ++k)
                if (picked[k].cigar == want) idx.push_back(k);
            if (idx.empty()) continue;
            ao.clear();
            bo.clear();
            al.clear();
            bl.clear();
            coff.assign(1, 0);
            for (uint32_t k : idx) {
                const DevReq &r = picked[k];
                ao.push_back(r.a_off);
                bo.push_back(r.b_off);
                al.push_back(r.m);
                bl.push_back(r.n);
                coff.push_back(coff.back() + (want ? nw_cigar_bound(r.m, r.n) : 0));
                cells += (uint64_t)r.m * r.n;
            }
            const uint32_t np = (uint32_t)idx.size();
            void *dsc = nullptr, *dcig = nullptr, *dlen = nullptr;
            int rc = scratch(ctx, "srv_scores", (size_t)np * 4 + 16, &dsc);
            if (!rc && want) rc = scratch(ctx, "srv_cigar", coff.back() + 16, &dcig);
            if (!rc && want) rc = scratch(ctx, "srv_cigar_len", (size_t)np * 8 + 16, &dlen);
            if (!rc) {
                const uint32_t fl = (want ? NW_CIGAR : 0u) | (srv->flags & (NW_LEARNED_BAND | NW_CIGAR_M));
                rc = nw_align_batch(ctx, srv->arena, ao.data(), al.data(), bo.data(), bl.data(), np, srv->sc, fl,
                                    (int32_t *)dsc, (char *)dcig, want ? coff.data() : nullptr, (uint64_t *)dlen);
            }
            scores.assign(np, 0);
            clen.assign(np, 0);
            cig.assign(want ? coff.back() + 1 : 1, 0);
            if (!rc) {
                cudaMemcpyAsync(scores.data(), dsc, (size_t)np * 4, cudaMemcpyDeviceToHost, ctx->stream);
                if (want) {
                    cudaMemcpyAsync(clen.data(), dlen, (size_t)np * 8, cudaMemcpyDeviceToHost, ctx->stream);
                    cudaMemcpyAsync(cig.data(), dcig, coff.back(), cudaMemcpyDeviceToHost, ctx->stream);
                }
                rc = nw_ctx_sync(ctx);
            }
            if (rc != NW_OK) {
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->failed_batches += 1;
                srv->last_error = std::string(nw_strerror(rc)) + ": " + nw_ctx_last_message(ctx) + " (" +
                                  std::to_string(np) + " requests)";
            }
            for (uint32_t q = 0; q < np; ++q) {
                Done &d = out[idx[q]];
                d.ticket = picked[idx[q]].ticket;
                d.status = rc;
                d.score = rc == NW_OK ? scores[q] : 0;
                if (want && rc == NW_OK) d.cigar.assign(cig.data() + coff[q], clen[q]);
            }
        }
        for (uint32_t k = 0; k < count; ++k) out[k].ticket = picked[k].ticket;
        // the reservation goes back on the device before anyone is told
        k_release<<<1, 32, 0, ctx->stream>>>(srv->dq, units);
        nw_ctx_sync(ctx);
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (uint32_t k = 0; k < count; ++k) {
                const uint64_t qi = picked[k].ticket - 1;  // queue index
                Live &lv = srv->live[qi - srv->live_front];
                lv.done = true;
                out[k].latency = t - lv.t_submit;
                srv->done.push_back(std::move(out[k]));
            }
            while (!srv->live.empty() && srv->live.front().done) {
                srv->live.pop_front();
                srv->live_front += 1;
            }
            srv->reserved -= (uint64_t)units * kUnit;
            srv->inflight -= count;
            srv->completed += count;
            srv->cells_done += cells;
            srv->batches += 1;
            srv->epoch += 1;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    cudaFree(d_out);
    cudaFreeHost(h_out);
}

// Publish `count` requests: place each one's bytes in the arena (a request
// never straddles the arena's end) and its descriptor in the next slot,
// waiting (bounded) while the arena or the ring is full of unfinished
// requests; copy them in with a few large copies on the intake stream; then
// make them visible to the workers.
template <typename Get>
static int enqueue(nw_server *srv, uint32_t count, Get get, uint64_t *tickets) {
    std::lock_guard<std::mutex> ik(srv->intake_mu);
    std::vector<uint8_t> stage;
    std::vector<DevReq> dstage;
    struct Seg {
        uint64_t dst, src, len;
    };
    std::vector<Seg> segs, dsegs;
    uint32_t k = 0;
    while (k < count) {
        uint32_t planned = 0;
        uint64_t first_q = 0;
        stage.clear();
        dstage.clear();
        segs.clear();
        dsegs.clear();
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop) return NW_ERR_ARG;
            first_q = srv->live_front + srv->live.size();
            const double t = now_s();
            while (k + planned < count && planned < (1u << 16) && stage.size() < (64u << 20)) {
                const uint8_t *a, *b;
                uint32_t m, n;
                bool cigar;
                get(k + planned, &a, &m, &b, &n, &cigar);
                const uint64_t la = (m + 3) / 4, lb = (n + 3) / 4;
                const uint64_t need = (la + 15) / 16 * 16 + (lb + 15) / 16 * 16;
                if (need > srv->arena_bytes) return NW_ERR_ARG;
                if (srv->live.empty())  // nothing in the arena: start over at its beginning
                    srv->arena_tail = (srv->arena_tail + srv->arena_bytes - 1) / srv->arena_bytes * srv->arena_bytes;
                uint64_t pos = srv->arena_tail;
                if (pos % srv->arena_bytes + need > srv->arena_bytes) pos += srv->arena_bytes - pos % srv->arena_bytes;
                const uint64_t front = srv->live.empty() ? srv->arena_tail : srv->live.front().start;
                const bool room = pos + need - front <= srv->arena_bytes && srv->live.size() < srv->slots;
                if (!room) {
                    if (planned > 0) break;  // publish what fits, then wait
                    const bool ok = srv->cv_done.wait_for(lk, std::chrono::seconds(60), [&] {
                        if (srv->stop || srv->live.empty()) return true;
                        uint64_t p = srv->arena_tail;
                        if (p % srv->arena_bytes + need > srv->arena_bytes) p += srv->arena_bytes - p % srv->arena_bytes;
                        return p + need - srv->live.front().start <= srv->arena_bytes && srv->live.size() < srv->slots;
                    });
                    if (!ok) return NW_ERR_TIMEOUT;
                    if (srv->stop) return NW_ERR_ARG;
                    continue;
                }
                const uint64_t phys = pos % srv->arena_bytes;
                const uint64_t src = stage.size();
                stage.resize(src + need, 0);
                memcpy(stage.data() + src, a, la);
                memcpy(stage.data() + src + (la + 15) / 16 * 16, b, lb);
                if (!segs.empty() && segs.back().dst + segs.back().len == phys) segs.back().len += need;
                else segs.push_back(Seg{phys, src, need});
                const uint64_t qi = first_q + planned;
                DevReq r{};
                r.a_off = phys;
                r.b_off = phys + (la + 15) / 16 * 16;
                r.ticket = qi + 1;
                r.m = m;
                r.n = n;
                r.units = (uint32_t)(trace_reserve(m, n, cigar) / kUnit);
                r.cigar = cigar ? 1u : 0u;
                const uint64_t slot = qi & (srv->slots - 1);
                if (!dsegs.empty() && dsegs.back().dst + dsegs.back().len == slot) dsegs.back().len += 1;
                else dsegs.push_back(Seg{slot, dstage.size(), 1});
                dstage.push_back(r);
                srv->live.push_back(Live{pos, t, false});
                srv->arena_tail = pos + need;
                if (tickets) tickets[k + planned] = r.ticket;
                ++planned;
            }
        }
        for (const Seg &s : segs)
            cudaMemcpyAsync(srv->arena + s.dst, stage.data() + s.src, s.len, cudaMemcpyHostToDevice, srv->intake);
        for (const Seg &s : dsegs)
            cudaMemcpyAsync(srv->ring + s.dst, dstage.data() + s.src, s.len * sizeof(DevReq), cudaMemcpyHostToDevice,
                            srv->intake);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            cudaEventRecord(srv->intake_ev, srv->intake);
            srv->tail += planned;
            srv->submitted += planned;
            srv->epoch += 1;
        }
        // (pageable sources: each copy has left `stage` when it returns)
        srv->cv_work.notify_all();
        k += planned;
    }
    return cudaGetLastError() == cudaSuccess ? NW_OK : NW_ERR_CUDA;
}

extern "C" {

nw_server *nw_server_create_ex(nw_ctx *ctx, uint32_t workers, uint32_t max_batch, uint64_t trace_budget,
                               uint64_t queue_bytes, uint32_t queue_slots, nw_scoring sc, uint32_t flags) {
    if (!ctx || workers == 0 || workers > 16 || max_batch == 0 || max_batch > (1u << 20)) return nullptr;
    if (queue_bytes < 4096 || queue_slots < 2 || (queue_slots & (queue_slots - 1)) || queue_slots > (1u << 30))
        return nullptr;
    if (check_scoring(ctx, sc) != NW_OK) return nullptr;
    if ((flags & NW_LEARNED_BAND) && sc.match < 2 * sc.gap) return nullptr;  // the certified band's bound needs it
    cudaSetDevice(ctx->device);
    nw_server *srv = new nw_server();
    srv->device = ctx->device;
    srv->sc = sc;
    srv->flags = flags;
    srv->budget = trace_budget;
    srv->budget_units = (uint32_t)std::min<uint64_t>(trace_budget / kUnit, 0xffffffffull);
    srv->max_batch = max_batch;
    srv->arena_bytes = (queue_bytes + 15) / 16 * 16;
    srv->slots = queue_slots;
    if (cudaMalloc(&srv->arena, srv->arena_bytes) != cudaSuccess ||
        cudaMalloc(&srv->ring, (size_t)queue_slots * sizeof(DevReq)) != cudaSuccess ||
        cudaMalloc(&srv->dq, sizeof(DevQueue)) != cudaSuccess || cudaMemset(srv->dq, 0, sizeof(DevQueue)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&srv->intake, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->intake_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(srv->intake_ev, srv->intake) != cudaSuccess) {
        cudaGetLastError();
        nw_server_destroy(srv);
        return nullptr;
    }
    // every worker gets its own context and stream; the learned model (if
    // the parent has one) is copied into each
    std::vector<float> params;
    if (ctx->band_model) {
        params.resize(nw_band_model_size());
        if (nw_band_model_get(ctx, params.data(), params.size()) != NW_OK) params.clear();
    }
    // each worker's scratch budget: a share of what is really available --
    // the creating context's unused budget, and at most 90 % of the device's
    // free memory (the creating context may hold scratch of earlier calls)
    size_t free_b = 0, total_b = 0;
    uint64_t avail = ctx->budget - std::min(ctx->budget, ctx->used);
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) avail = std::min<uint64_t>(avail, (uint64_t)(free_b * 0.9));
    else cudaGetLastError();
    const uint64_t per = avail / (workers + 1);
    for (uint32_t w = 0; w < workers; ++w) {
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

nw_server *nw_server_create(nw_ctx *ctx, uint32_t workers, uint32_t max_batch, uint64_t trace_budget, nw_scoring sc,
                            uint32_t flags) {
    return nw_server_create_ex(ctx, workers, max_batch, trace_budget, 1ull << 30, 1u << 20, sc, flags);
}

int nw_server_submit(nw_server *srv, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                     uint32_t want_cigar, uint64_t *ticket) {
    if (!srv || (m && !a2b) || (n && !b2b)) return NW_ERR_ARG;
    if (m >= (1u << 30) || n >= (1u << 30)) return NW_ERR_ARG;
    return enqueue(
        srv, 1u,
        [&](uint32_t, const uint8_t **a, uint32_t *mm, const uint8_t **b, uint32_t *nn, bool *c) {
            *a = a2b;
            *mm = m;
            *b = b2b;
            *nn = n;
            *c = want_cigar != 0;
        },
        ticket);
}

int nw_server_submit_many(nw_server *srv, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                          const uint64_t *b_off, const uint32_t *b_len, const uint8_t *want_cigar, uint32_t count,
                          uint64_t *tickets) {
    if (!srv || (count && (!pool2b || !a_off || !a_len || !b_off || !b_len || !want_cigar))) return NW_ERR_ARG;
    for (uint32_t k = 0; k < count; ++k)
        if (a_len[k] >= (1u << 30) || b_len[k] >= (1u << 30)) return NW_ERR_ARG;
    return enqueue(
        srv, count,
        [&](uint32_t k, const uint8_t **a, uint32_t *m, const uint8_t **b, uint32_t *n, bool *c) {
            *a = pool2b + a_off[k];
            *m = a_len[k];
            *b = pool2b + b_off[k];
            *n = b_len[k];
            *c = want_cigar[k] != 0;
        },
        tickets);
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

int64_t nw_server_last_message(nw_server *srv, char *buf, uint64_t cap) {
    if (!srv || (cap && !buf)) return -NW_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t len = srv->last_error.size();
    if (cap) {
        const uint64_t k = std::min<uint64_t>(len, cap - 1);
        memcpy(buf, srv->last_error.data(), k);
        buf[k] = '\0';
    }
    return (int64_t)len;
}

int nw_server_drain(nw_server *srv, double timeout_s) {
    if (!srv) return NW_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                          [&] { return srv->tail == srv->head_host && srv->inflight == 0; });
    return ok ? NW_OK : NW_ERR_TIMEOUT;
}

int nw_server_stats(nw_server *srv, uint64_t *out, int cap) {
    if (!srv || !out) return -NW_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t v[8] = {srv->submitted, srv->completed, srv->tail - srv->head_host, srv->inflight,
                           srv->cells_done, srv->reserved, srv->batches, srv->budget};
    for (int k = 0; k < cap && k < 8; ++k) out[k] = v[k];
    return 8;
}

int nw_server_queue_state(nw_server *srv, uint64_t *admitted, uint64_t *reserved_bytes) {
    if (!srv || !admitted || !reserved_bytes) return NW_ERR_ARG;
    cudaSetDevice(srv->device);
    DevQueue q{};
    {
        std::lock_guard<std::mutex> ik(srv->intake_mu);
        if (cudaMemcpyAsync(&q, srv->dq, sizeof(q), cudaMemcpyDeviceToHost, srv->intake) != cudaSuccess ||
            cudaStreamSynchronize(srv->intake) != cudaSuccess) {
            cudaGetLastError();
            return NW_ERR_CUDA;
        }
    }
    *admitted = q.state >> 32;
    *reserved_bytes = (q.state & 0xffffffffull) * kUnit;
    return NW_OK;
}

void nw_server_destroy(nw_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (auto &t : srv->workers)
        if (t.joinable()) t.join();
    for (nw_ctx *c : srv->ctxs) {
        cudaStream_t st = c->stream;
        nw_ctx_destroy(c);
        if (st) cudaStreamDestroy(st);
    }
    if (srv->intake) cudaStreamSynchronize(srv->intake);
    if (srv->intake_ev) cudaEventDestroy(srv->intake_ev);
    if (srv->intake) cudaStreamDestroy(srv->intake);
    if (srv->arena) cudaFree(srv->arena);
    if (srv->ring) cudaFree(srv->ring);
    if (srv->dq) cudaFree(srv->dq);
    delete srv;
}

}  // extern "C"
