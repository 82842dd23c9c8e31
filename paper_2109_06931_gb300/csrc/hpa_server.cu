// Serving: a request loop over sample buffers as they arrive (the serving
// analogue of streaming aggregation over profiles, Section 6.1).
//
// One worker thread owns the handle.  Requests wait in a FIFO queue; they are
// admitted while their device bytes (samples in, keys out) fit in a ring of
// mem_cap_bytes that the server reserves once, so admission is by free device
// memory and no allocation happens per request.  Whatever has been admitted
// when the GPU can take more work forms the next batch (up to max_batch
// requests): its inputs are copied on a copy stream, its aggregation runs as
// one batched call on the handle's stream, and its keys are copied back on a
// second copy stream, so the copies of one batch overlap the kernels of the
// next.  Batches retire in order; latency is measured from submit to the
// moment the host arrays hold the result.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hpa_host.h"

using namespace hpa;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t SLOT_WORDS = 1 + 2 * HPA_MAX_STALL;

struct Req {
    uint64_t ticket = 0;
    uint32_t bin = 0;
    hpa_samples in{};       // host arrays
    hpa_profile out{};      // host arrays
    double t_submit = 0, t_done = 0;
    size_t bytes = 0, off = 0;
    hpa_samples din{};      // device copies (in the ring)
    hpa_profile dout{};
    uint64_t* h_nkeys = nullptr;   // pinned slot: n_keys, then totals and UNKNOWN totals
    hpa_status status = HPA_OK;
    bool done = false;
};

struct Batch {
    std::vector<Req*> reqs;
    cudaEvent_t in_done = nullptr, computed = nullptr, copied = nullptr;
    // stage timing: copy-in start, compute start and end, copy-out start
    cudaEvent_t in0 = nullptr, c0 = nullptr, c1 = nullptr, out0 = nullptr;
    double launch_s = 0;
    int stage = 0;          // 0 computing, 1 copying keys out

};

}  // namespace

struct hpa_server {
    hpa_handle* h = nullptr;
    hpa_server_options opt{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    std::deque<Batch*> inflight;
    uint64_t next_ticket = 1;
    bool stop = false;
    // device ring (FIFO allocation)
    char* ring = nullptr;
    size_t ring_cap = 0, ring_head = 0;
    // copy_meta carries the small result copies (key counts), so that a
    // batch's count is known as soon as it is computed instead of behind the
    // previous batch's keys on copy_out
    cudaStream_t copy_in = nullptr, copy_out = nullptr, copy_meta = nullptr;
    // pinned slots of SLOT_WORDS words (n_keys, totals, UNKNOWN totals): the
    // small results land here, so that no copy targets pageable host memory
    // (such a copy would block the worker until the copy stream reaches it)
    uint64_t* pinned = nullptr;
    size_t pinned_cap = 0, pinned_next = 0;
    // stats
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, rejected = 0, samples_done = 0, batches = 0;
    double stage_ms[5] = {0, 0, 0, 0, 0}, launch_ms = 0;
    uint64_t timed_batches = 0;
    double t_first = 0, t_last = 0;
    std::string err;

    // FIFO ring: requests are allocated and released in the same order.
    // live holds (offset, bytes) of every live request, oldest first; while
    // `wrapped`, head lies in the ring's start and the oldest entries at its end.
    std::deque<std::pair<size_t, size_t>> live;
    bool wrapped = false;
    bool ring_alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes > ring_cap) return false;
        if (live.empty()) { ring_head = 0; wrapped = false; }
        const size_t oldest = live.empty() ? 0 : live.front().first;
        if (!wrapped) {
            if (ring_head + bytes <= ring_cap) { *off = ring_head; ring_head += bytes; }
            else if (!live.empty() && bytes <= oldest) { *off = 0; ring_head = bytes; wrapped = true; }
            else return false;
        } else {
            if (ring_head + bytes <= oldest) { *off = ring_head; ring_head += bytes; }
            else return false;
        }
        live.push_back({*off, bytes});
        return true;
    }
    void ring_release(size_t n) {
        for (size_t i = 0; i < n && !live.empty(); ++i) {
            const size_t before = live.front().first;
            live.pop_front();
            if (live.empty()) { wrapped = false; ring_head = 0; }
            else if (wrapped && live.front().first < before) wrapped = false;
        }
    }
    void loop();
    void retire();
    bool admit_and_launch();
};

static size_t req_bytes(const hpa_samples& s, uint64_t cap) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t b = al(s.n * 8) + al(s.n * 4) + al(s.n) + (s.count ? al(s.n * 4) : 0);
    b += al(cap * 4) + al(cap * 4) + al(cap) + al(cap * 8) + al(8) + 2 * al(8 * HPA_MAX_STALL);
    return b;
}

void hpa_server::retire() {
    while (!inflight.empty()) {
        Batch* b = inflight.front();
        if (b->stage == 0) {
            if (cudaEventQuery(b->computed) != cudaSuccess) { cudaGetLastError(); return; }
            // keys are known: copy exactly K of them for every request
            cudaEventRecord(b->out0, copy_out);
            for (Req* r : b->reqs) {
                const uint64_t K = std::min<uint64_t>(*r->h_nkeys, r->out.capacity);
                if (K) {
                    cudaMemcpyAsync(r->out.key_ctx, r->dout.key_ctx, K * 4, cudaMemcpyDeviceToHost, copy_out);
                    cudaMemcpyAsync(r->out.key_node, r->dout.key_node, K * 4, cudaMemcpyDeviceToHost, copy_out);
                    cudaMemcpyAsync(r->out.key_stall, r->dout.key_stall, K, cudaMemcpyDeviceToHost, copy_out);
                    cudaMemcpyAsync(r->out.val, r->dout.val, K * 8, cudaMemcpyDeviceToHost, copy_out);
                }
                if (r->out.total) cudaMemcpyAsync(r->h_nkeys + 1, r->dout.total, 8 * r->in.n_stall, cudaMemcpyDeviceToHost, copy_out);
                if (r->out.unknown)
                    cudaMemcpyAsync(r->h_nkeys + 1 + HPA_MAX_STALL, r->dout.unknown, 8 * r->in.n_stall,
                                    cudaMemcpyDeviceToHost, copy_out);
            }
            cudaEventRecord(b->copied, copy_out);
            b->stage = 1;
        }
        if (cudaEventQuery(b->copied) != cudaSuccess) { cudaGetLastError(); return; }
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lock(mu);
            for (Req* r : b->reqs) {
                *r->out.n_keys = *r->h_nkeys;
                if (r->out.total) std::memcpy(r->out.total, r->h_nkeys + 1, 8 * r->in.n_stall);
                if (r->out.unknown) std::memcpy(r->out.unknown, r->h_nkeys + 1 + HPA_MAX_STALL, 8 * r->in.n_stall);
                if (r->status == HPA_OK && *r->h_nkeys > r->out.capacity) r->status = HPA_E_CAPACITY;
                r->t_done = t;
                r->done = true;
                lat.push_back((t - r->t_submit) * 1e3);
                samples_done += r->in.n;
                ++completed;
            }
            t_last = t;
            ring_release(b->reqs.size());
        }
        {
            float ms[5] = {0, 0, 0, 0, 0};
            cudaEventElapsedTime(&ms[0], b->in0, b->in_done);
            cudaEventElapsedTime(&ms[1], b->in_done, b->c0);
            cudaEventElapsedTime(&ms[2], b->c0, b->c1);
            cudaEventElapsedTime(&ms[3], b->c1, b->out0);
            cudaEventElapsedTime(&ms[4], b->out0, b->copied);
            cudaGetLastError();
            std::lock_guard<std::mutex> lock(mu);
            for (int i = 0; i < 5; ++i) stage_ms[i] += ms[i];
            launch_ms += b->launch_s * 1e3;
            ++timed_batches;
        }
        done_cv.notify_all();
        for (cudaEvent_t e : {b->in_done, b->computed, b->copied, b->in0, b->c0, b->c1, b->out0}) cudaEventDestroy(e);
        delete b;
        inflight.pop_front();
    }
}

bool hpa_server::admit_and_launch() {
    std::vector<Req*> take;
    {
        std::lock_guard<std::mutex> lock(mu);
        while (!queue.empty() && take.size() < opt.max_batch) {
            Req* r = queue.front();
            if (r->bytes > ring_cap) {            // can never fit
                r->status = HPA_E_OOM;
                r->done = true;
                ++rejected;
                queue.pop_front();
                continue;
            }
            size_t off;
            if (!ring_alloc(r->bytes, &off)) break;
            r->off = off;
            queue.pop_front();
            take.push_back(r);
        }
        if (!take.empty() && t_first == 0) t_first = now_s();
    }
    done_cv.notify_all();
    if (take.empty()) return false;
    Trace trace_("hpa.server.batch");
    const double t_admit = now_s();
    Batch* b = new Batch();
    b->reqs = take;
    for (cudaEvent_t* e : {&b->in_done, &b->computed, &b->copied, &b->in0, &b->c0, &b->c1, &b->out0})
        cudaEventCreate(e);
    cudaEventRecord(b->in0, copy_in);
    std::vector<uint32_t> ids;
    std::vector<hpa_samples> ins;
    std::vector<hpa_profile> outs;
    for (Req* r : take) {
        Carve c{ring + r->off};
        const hpa_samples& s = r->in;
        const uint64_t cap = std::min<uint64_t>(r->out.capacity, s.n ? s.n : 1);
        r->din = s;
        r->din.pc = c.take<uint64_t>(s.n);
        r->din.ctx = c.take<uint32_t>(s.n);
        r->din.stall = c.take<uint8_t>(s.n);
        r->din.count = s.count ? c.take<uint32_t>(s.n) : nullptr;
        r->dout = r->out;
        r->dout.capacity = cap;
        r->dout.key_ctx = c.take<uint32_t>(cap);
        r->dout.key_node = c.take<uint32_t>(cap);
        r->dout.key_stall = c.take<uint8_t>(cap);
        r->dout.val = c.take<uint64_t>(cap);
        r->dout.n_keys = c.take<uint64_t>(1);
        r->dout.total = c.take<uint64_t>(HPA_MAX_STALL);
        r->dout.unknown = c.take<uint64_t>(HPA_MAX_STALL);
        cudaMemcpyAsync((void*)r->din.pc, s.pc, s.n * 8, cudaMemcpyHostToDevice, copy_in);
        cudaMemcpyAsync((void*)r->din.ctx, s.ctx, s.n * 4, cudaMemcpyHostToDevice, copy_in);
        cudaMemcpyAsync((void*)r->din.stall, s.stall, s.n, cudaMemcpyHostToDevice, copy_in);
        if (s.count) cudaMemcpyAsync((void*)r->din.count, s.count, s.n * 4, cudaMemcpyHostToDevice, copy_in);
        r->h_nkeys = pinned + (pinned_next++ % pinned_cap) * SLOT_WORDS;
        ids.push_back(r->bin);
        ins.push_back(r->din);
        outs.push_back(r->dout);
    }
    cudaEventRecord(b->in_done, copy_in);
    cudaStreamWaitEvent(h->stream, b->in_done, 0);
    cudaEventRecord(b->c0, h->stream);
    hpa_status st = h->aggregate((uint32_t)take.size(), ids.data(), ins.data(), outs.data(), false);
    cudaEventRecord(b->c1, h->stream);
    if (st) {
        std::lock_guard<std::mutex> lock(mu);
        err = h->err;
        for (Req* r : take) r->status = st;
    }
    cudaEventRecord(b->computed, h->stream);
    cudaStreamWaitEvent(copy_meta, b->computed, 0);
    for (size_t i = 0; i < take.size(); ++i)
        cudaMemcpyAsync(take[i]->h_nkeys, outs[i].n_keys, 8, cudaMemcpyDeviceToHost, copy_meta);
    // the computed event must be after the n_keys copies for retire() to read them
    cudaEventRecord(b->computed, copy_meta);
    ++batches;
    b->launch_s = now_s() - t_admit;
    inflight.push_back(b);
    return true;
}

void hpa_server::loop() {
    cudaSetDevice(h->device);
    while (true) {
        retire();
        const bool launched = inflight.size() < opt.max_inflight && admit_and_launch();
        std::unique_lock<std::mutex> lock(mu);
        if (stop && queue.empty() && inflight.empty()) break;
        if (!launched) {
            if (inflight.empty()) cv.wait_for(lock, std::chrono::milliseconds(5));
            else {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
        }
    }
}

extern "C" hpa_status hpa_server_create(hpa_handle* h, const hpa_server_options* opt, hpa_server** out) {
    if (!h || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    hpa_server* s = new hpa_server();
    s->h = h;
    if (opt) s->opt = *opt;
    if (!s->opt.mem_cap_bytes) s->opt.mem_cap_bytes = 60ull << 30;
    if (!s->opt.max_batch) s->opt.max_batch = 64;
    if (!s->opt.max_inflight) s->opt.max_inflight = 3;
    s->ring_cap = s->opt.mem_cap_bytes;
    // more slots than requests can be in flight
    s->pinned_cap = std::max<size_t>(4096, 2 * (size_t)s->opt.max_batch * (s->opt.max_inflight + 1));
    const unsigned long long cap_bytes = s->opt.mem_cap_bytes;
    if (cudaMalloc((void**)&s->ring, s->ring_cap) != cudaSuccess ||
        cudaMallocHost((void**)&s->pinned, s->pinned_cap * SLOT_WORDS * 8) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_meta, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (s->ring) cudaFree(s->ring);
        if (s->pinned) cudaFreeHost(s->pinned);
        delete s;
        return h->fail(HPA_E_OOM, "server: cannot reserve %llu bytes of device memory", cap_bytes);
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return HPA_OK;
}

extern "C" hpa_status hpa_server_submit(hpa_server* s, uint32_t binary_id, const hpa_samples* in, hpa_profile* out,
                                        uint64_t* ticket) {
    if (!s || !in || !out || !ticket) return HPA_E_INVALID_ARG;
    if (!s->h->binary(binary_id)) return HPA_E_INVALID_ARG;
    if (in->n && (!in->pc || !in->ctx || !in->stall)) return HPA_E_INVALID_ARG;
    if (!out->n_keys || (out->capacity && (!out->key_ctx || !out->key_node || !out->key_stall || !out->val)))
        return HPA_E_INVALID_ARG;
    Req* r = new Req();
    r->bin = binary_id;
    r->in = *in;
    r->out = *out;
    r->bytes = req_bytes(*in, std::min<uint64_t>(out->capacity, in->n ? in->n : 1));
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        ++s->submitted;
    }
    s->cv.notify_one();
    *ticket = r->ticket;
    return HPA_OK;
}

extern "C" hpa_status hpa_server_poll(hpa_server* s, uint64_t ticket, int wait_ms) {
    if (!s) return HPA_E_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HPA_E_INVALID_ARG;
    Req* r = it->second;
    if (!r->done && wait_ms > 0)
        s->done_cv.wait_for(lock, std::chrono::milliseconds(wait_ms), [r] { return r->done; });
    if (!r->done) return HPA_PENDING;
    const hpa_status st = r->status;
    s->reqs.erase(it);
    delete r;
    return st;
}

extern "C" hpa_status hpa_server_stats_get(hpa_server* s, hpa_server_stats* st) {
    if (!s || !st) return HPA_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *st = hpa_server_stats{};
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->samples = s->samples_done;
    st->batches = s->batches;
    st->busy_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        st->p50_ms = q(0.50);
        st->p99_ms = q(0.99);
        st->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
    }
    if (s->timed_batches) {
        const double k = 1.0 / (double)s->timed_batches;
        st->h2d_ms = s->stage_ms[0] * k;
        st->wait_compute_ms = s->stage_ms[1] * k;
        st->compute_ms = s->stage_ms[2] * k;
        st->wait_d2h_ms = s->stage_ms[3] * k;
        st->d2h_ms = s->stage_ms[4] * k;
        st->launch_ms = s->launch_ms * k;
    }
    return HPA_OK;
}

extern "C" hpa_status hpa_server_destroy(hpa_server* s) {
    if (!s) return HPA_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->h->device);
    cudaStreamSynchronize(s->copy_in);
    cudaStreamSynchronize(s->copy_out);
    cudaStreamSynchronize(s->copy_meta);
    cudaStreamDestroy(s->copy_in);
    cudaStreamDestroy(s->copy_out);
    cudaStreamDestroy(s->copy_meta);
    cudaFree(s->ring);
    cudaFreeHost(s->pinned);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return HPA_OK;
}
