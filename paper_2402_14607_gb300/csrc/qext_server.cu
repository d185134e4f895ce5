// Serving loop: continuous batching of extraction requests from many QRNG
// channels (stream pairs), each with its own plan (n, q, m) and chaining
// state kept on the device.
//
// A request carries one piece of a channel's raw streams (packed words, or
// b-bit ADC samples) in host memory and a host buffer for its output: the
// m-bit outputs of the blocks it completes, concatenated (Algorithm 1's
// output order; a block straddling requests completes in the later one).
// Requests of one channel run one at a time in arrival order; requests of
// different channels run together.
//
// The scheduler thread loops over:
//   completions  rounds whose device->host copy finished: record latency,
//                free their device memory, release their channels;
//   admission    the oldest request of each idle channel, in arrival order,
//                if its device memory fits the arena (the HBM budget);
//                host->device copies start at once on the copy-in stream;
//   rounds       admitted requests form a round on the compute stream (it
//                waits on their copies): ingest kernels for sample input,
//                ONE batched extraction launch for requests that start and
//                end on block boundaries of a channel with no carried tail,
//                a stream push for the others; the outputs return on the
//                copy-out stream.
// New requests are admitted while earlier rounds run, so copies and kernels
// of consecutive rounds overlap.  With a fake executor no GPU is touched:
// requests complete as soon as their round forms (host logic tests).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "qext_internal.h"
#include "qext_nvtx.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::time_point t) {
    return std::chrono::duration<double>(t.time_since_epoch()).count();
}

// First-fit allocator over [0, size) in 256-byte units (offsets only; the
// device base pointer is added by the caller).
class Arena {
public:
    explicit Arena(uint64_t size) : size_(size & ~uint64_t(255)) {
        if (size_) free_[0] = size_;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = (bytes + 255) & ~uint64_t(255);
        if (!bytes) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + 255) & ~uint64_t(255);
        if (!bytes) bytes = 256;
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
    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }

private:
    uint64_t size_, used_ = 0, peak_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

struct Request {
    uint64_t id = 0;
    uint32_t channel = 0;
    uint32_t b = 0;        // 0: packed words, else bits per sample
    const void *hx = nullptr, *hy = nullptr;
    uint64_t count = 0;    // samples (b > 0) or stream bits (b == 0)
    uint64_t nbits = 0;    // stream bits of each source
    uint32_t *hout = nullptr;
    uint64_t out_cap = 0;  // words
    uint64_t in_bytes = 0, words = 0, out_words = 0;
    uint64_t blocks = 0, out_bits = 0;
    uint64_t off = 0, bytes = 0;  // arena allocation
    bool batched = false;
    int status = QEXT_OK;
    Clock::time_point t_submit, t_done;
    cudaEvent_t h2d = nullptr;
};

struct Channel {
    const qext_plan *plan = nullptr;
    qext_stream *stream = nullptr;  // device chaining state (tails)
    std::deque<Request *> queue;
    bool busy = false;
    uint64_t host_tail = 0;  // tail bits (fake executor bookkeeping)
};

struct Round {
    std::vector<Request *> reqs;
    cudaEvent_t done = nullptr;  // outputs are back on the host
    int stage = -1;              // staging buffer in use (-1: none)
};

}  // namespace

struct qext_server {
    qext_server_config cfg;
    Arena arena{0};
    uint8_t *dbase = nullptr;
    std::vector<Channel> channels;
    std::deque<Request *> arrivals;  // submitted, not yet admitted (arrival order)
    std::vector<Request *> admitted;  // copies issued, waiting for a round
    std::deque<Round> inflight;
    std::vector<qext_completion> completions;
    std::mutex mu;
    std::condition_variable cv;
    std::thread thread;
    bool stop = false;
    uint64_t next_id = 1;
    qext_server_stats stats{};
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    void *d_table[2] = {nullptr, nullptr};
    void *h_stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    int next_stage = 0;
    int device = 0;
};

namespace {

uint64_t out_words_for(uint64_t bits) { return (bits + 31) / 32; }

// bytes of device memory a request needs: raw inputs, packed words (sample
// input only), output
uint64_t request_bytes(const Request &r) {
    uint64_t b = 2 * ((r.in_bytes + 255) & ~uint64_t(255));
    if (r.b) b += 2 * ((r.words * 4 + 255) & ~uint64_t(255));
    return b + ((r.out_words * 4 + 255) & ~uint64_t(255)) + 256;
}

void finish(qext_server *S, Request *r, int status) {
    r->status = status;
    r->t_done = Clock::now();
    Channel &ch = S->channels[r->channel];
    ch.busy = false;
    if (r->bytes) S->arena.release(r->off, r->bytes);
    if (r->h2d) cudaEventDestroy(r->h2d);
    qext_completion c;
    std::memset(&c, 0, sizeof c);
    c.request_id = r->id;
    c.channel = r->channel;
    c.status = status;
    c.out_bits = r->out_bits;
    c.blocks = r->blocks;
    c.submit_s = seconds(r->t_submit);
    c.done_s = seconds(r->t_done);
    c.latency_s = c.done_s - c.submit_s;
    c.batched = r->batched ? 1 : 0;
    S->completions.push_back(c);
    S->stats.completed++;
    S->stats.bits_out += r->out_bits;
    delete r;
}

// device pointers of a request's pieces inside the arena
struct Bufs {
    uint8_t *rx, *ry;
    uint32_t *px, *py, *out;
};

Bufs bufs_of(qext_server *S, const Request &r) {
    uint8_t *p = S->dbase + r.off;
    const uint64_t raw = (r.in_bytes + 255) & ~uint64_t(255);
    const uint64_t pk = (r.words * 4 + 255) & ~uint64_t(255);
    Bufs b;
    b.rx = p;
    b.ry = p + raw;
    if (r.b) {
        b.px = reinterpret_cast<uint32_t *>(p + 2 * raw);
        b.py = reinterpret_cast<uint32_t *>(p + 2 * raw + pk);
        b.out = reinterpret_cast<uint32_t *>(p + 2 * raw + 2 * pk);
    } else {
        b.px = reinterpret_cast<uint32_t *>(b.rx);
        b.py = reinterpret_cast<uint32_t *>(b.ry);
        b.out = reinterpret_cast<uint32_t *>(p + 2 * raw);
    }
    return b;
}

// Admission: oldest requests first, one per idle channel, within the budget.
void admit(qext_server *S) {
    for (auto it = S->arrivals.begin(); it != S->arrivals.end();) {
        Request *r = *it;
        Channel &ch = S->channels[r->channel];
        if (ch.busy || ch.queue.empty() || ch.queue.front() != r) {
            ++it;
            continue;
        }
        const uint64_t need = request_bytes(*r);
        uint64_t off = 0;
        if (!S->arena.alloc(need, &off)) {
            ++it;  // waits for memory; later, smaller requests of other channels may still fit
            continue;
        }
        r->off = off;
        r->bytes = need;
        ch.busy = true;
        ch.queue.pop_front();
        it = S->arrivals.erase(it);
        if (!S->cfg.fake_executor) {
            const Bufs b = bufs_of(S, *r);
            cudaEventCreateWithFlags(&r->h2d, cudaEventDisableTiming);
            if (cudaMemcpyAsync(b.rx, r->hx, r->in_bytes, cudaMemcpyHostToDevice, S->s_in) != cudaSuccess ||
                cudaMemcpyAsync(b.ry, r->hy, r->in_bytes, cudaMemcpyHostToDevice, S->s_in) != cudaSuccess ||
                cudaEventRecord(r->h2d, S->s_in) != cudaSuccess) {
                finish(S, r, QEXT_E_CUDA);
                continue;
            }
        }
        S->admitted.push_back(r);
    }
}

// A round: everything admitted so far, up to max_batch requests.
void launch_round(qext_server *S) {
    if (S->admitted.empty()) return;
    Round rd;
    const size_t take = std::min<size_t>(S->admitted.size(), S->cfg.max_batch);
    rd.reqs.assign(S->admitted.begin(), S->admitted.begin() + take);
    S->admitted.erase(S->admitted.begin(), S->admitted.begin() + take);
    S->stats.rounds++;
    S->stats.max_round = std::max<uint64_t>(S->stats.max_round, rd.reqs.size());
    if (S->cfg.fake_executor) {
        for (Request *r : rd.reqs) {
            Channel &ch = S->channels[r->channel];
            const uint64_t v = ch.host_tail + r->nbits;
            r->blocks = v / ch.plan->n;
            r->batched = ch.host_tail == 0 && r->nbits % ch.plan->n == 0;
            ch.host_tail = v - r->blocks * ch.plan->n;
            r->out_bits = r->blocks * ch.plan->m;
            finish(S, r, QEXT_OK);
        }
        return;
    }
    std::vector<qext_batch_item> items;
    for (Request *r : rd.reqs) {
        Channel &ch = S->channels[r->channel];
        const Bufs b = bufs_of(S, *r);
        cudaStreamWaitEvent(S->s_comp, r->h2d, 0);
        int rc = QEXT_OK;
        if (r->b) {
            rc = qext_pack_samples(r->b, reinterpret_cast<const uint16_t *>(b.rx), r->count, b.px,
                                   reinterpret_cast<qext_cuda_stream>(S->s_comp));
            if (rc == QEXT_OK)
                rc = qext_pack_samples(r->b, reinterpret_cast<const uint16_t *>(b.ry), r->count, b.py,
                                       reinterpret_cast<qext_cuda_stream>(S->s_comp));
        }
        const uint64_t n = ch.plan->n;
        if (rc == QEXT_OK && ch.stream->tail_bits == 0 && r->nbits % n == 0) {
            r->blocks = r->nbits / n;
            r->batched = true;
            ch.stream->blocks_done += r->blocks;
            if (r->blocks) items.push_back(qext_batch_item{ch.plan, b.px, b.py, r->blocks, b.out});
        } else if (rc == QEXT_OK) {
            // carried tail or a partial block: the stream path (general kernel)
            const uint64_t t = ch.stream->tail_bits;
            r->blocks = (t + r->nbits) / n;
            uint64_t w = 0;
            rc = qext_stream_push(ch.stream, b.px, b.py, r->nbits, b.out, r->out_words, &w,
                                  reinterpret_cast<qext_cuda_stream>(S->s_comp));
            ch.stream->pending_bits = 0;  // each request returns its own bit string
        }
        r->out_bits = r->blocks * ch.plan->m;
        if (rc != QEXT_OK) r->status = rc;
    }
    if (!items.empty()) {
        const qext::NvtxRange range("qext serving round (batched launch)");
        const int st = S->next_stage;
        S->next_stage ^= 1;
        cudaEventSynchronize(S->stage_free[st]);  // the staging copy of two rounds ago
        const int rc = qext::batch_launch_tables(items.data(), uint32_t(items.size()), S->d_table[st], S->h_stage[st],
                                                 reinterpret_cast<qext_cuda_stream>(S->s_comp));
        cudaEventRecord(S->stage_free[st], S->s_comp);
        if (rc != QEXT_OK)
            for (Request *r : rd.reqs)
                if (r->batched) r->status = rc;
    }
    cudaEvent_t comp;
    cudaEventCreateWithFlags(&comp, cudaEventDisableTiming);
    cudaEventRecord(comp, S->s_comp);
    cudaStreamWaitEvent(S->s_out, comp, 0);
    cudaEventDestroy(comp);
    for (Request *r : rd.reqs) {
        const uint64_t ow = out_words_for(r->out_bits);
        if (ow && r->status == QEXT_OK)
            cudaMemcpyAsync(r->hout, bufs_of(S, *r).out, ow * 4, cudaMemcpyDeviceToHost, S->s_out);
    }
    cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming);
    cudaEventRecord(rd.done, S->s_out);
    S->inflight.push_back(std::move(rd));
}

void complete_rounds(qext_server *S) {
    while (!S->inflight.empty()) {
        Round &rd = S->inflight.front();
        const cudaError_t e = cudaEventQuery(rd.done);
        if (e == cudaErrorNotReady) break;
        for (Request *r : rd.reqs) finish(S, r, e == cudaSuccess ? r->status : QEXT_E_CUDA);
        cudaEventDestroy(rd.done);
        S->inflight.pop_front();
    }
}

void loop(qext_server *S) {
    if (!S->cfg.fake_executor) cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop || !S->arrivals.empty() || !S->admitted.empty() || !S->inflight.empty()) {
        complete_rounds(S);
        admit(S);
        launch_round(S);
        S->stats.bytes_in_use = S->arena.used();
        S->stats.peak_bytes = S->arena.peak();
        S->cv.notify_all();
        const bool idle = S->admitted.empty();
        if (idle) S->cv.wait_for(lk, std::chrono::microseconds(S->inflight.empty() ? 500 : 20));
    }
}

}  // namespace

extern "C" {

int qext_server_create(const qext_server_config *cfg, qext_server **out) {
    if (!cfg || !out || cfg->max_batch == 0 || cfg->max_batch > QEXT_NOALLOC_MAX_ITEMS || cfg->hbm_budget_bytes < 4096)
        return QEXT_E_INVAL;
    *out = nullptr;
    qext_server *S = new (std::nothrow) qext_server();
    if (!S) return QEXT_E_INVAL;
    S->cfg = *cfg;
    S->arena = Arena(cfg->hbm_budget_bytes);
    if (!cfg->fake_executor) {
        bool ok = cudaGetDevice(&S->device) == cudaSuccess &&
                  cudaMalloc(reinterpret_cast<void **>(&S->dbase), S->arena.size()) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&S->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; ok && i < 2; ++i)
            ok = cudaMalloc(&S->d_table[i], qext::batch_table_bytes()) == cudaSuccess &&
                 cudaHostAlloc(&S->h_stage[i], qext::batch_table_bytes(), cudaHostAllocDefault) == cudaSuccess &&
                 cudaEventCreateWithFlags(&S->stage_free[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventRecord(S->stage_free[i], S->s_comp) == cudaSuccess;
        if (!ok) {
            qext_server_destroy(S);
            return QEXT_E_CUDA;
        }
    }
    S->thread = std::thread(loop, S);
    *out = S;
    return QEXT_OK;
}

int qext_server_destroy(qext_server *S) {
    if (!S) return QEXT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->thread.joinable()) S->thread.join();
    for (Channel &ch : S->channels)
        if (ch.stream) qext_stream_destroy(ch.stream);
    if (!S->cfg.fake_executor) {
        for (int i = 0; i < 2; ++i) {
            if (S->stage_free[i]) cudaEventDestroy(S->stage_free[i]);
            cudaFree(S->d_table[i]);
            if (S->h_stage[i]) cudaFreeHost(S->h_stage[i]);
        }
        if (S->s_in) cudaStreamDestroy(S->s_in);
        if (S->s_comp) cudaStreamDestroy(S->s_comp);
        if (S->s_out) cudaStreamDestroy(S->s_out);
        cudaFree(S->dbase);
    }
    delete S;
    return QEXT_OK;
}

int qext_server_add_channel(qext_server *S, const qext_plan *p, uint32_t *channel) {
    if (!S || !p || !channel) return QEXT_E_INVAL;
    if (!p->gpu_supported) return QEXT_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(S->mu);
    Channel ch;
    ch.plan = p;
    if (!S->cfg.fake_executor) {
        cudaSetDevice(S->device);
        const int rc = qext_stream_create(p, &ch.stream);
        if (rc != QEXT_OK) return rc;
    }
    *channel = uint32_t(S->channels.size());
    S->channels.push_back(std::move(ch));
    return QEXT_OK;
}

int qext_server_submit(qext_server *S, uint32_t channel, uint32_t b, const void *x_host, const void *y_host,
                       uint64_t count, uint32_t *out_host, uint64_t out_capacity_words, uint64_t *request_id) {
    if (!S || !request_id) return QEXT_E_INVAL;
    *request_id = 0;
    if (b > 16 || count == 0 || (!S->cfg.fake_executor && (!x_host || !y_host))) return QEXT_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (channel >= S->channels.size()) return QEXT_E_INVAL;
    Channel &ch = S->channels[channel];
    Request *r = new (std::nothrow) Request();
    if (!r) return QEXT_E_INVAL;
    r->channel = channel;
    r->b = b;
    r->hx = x_host;
    r->hy = y_host;
    r->count = count;
    r->nbits = b ? count * b : count;
    r->words = (r->nbits + 31) / 32;
    r->in_bytes = b ? count * 2 : r->words * 4;
    r->hout = out_host;
    r->out_cap = out_capacity_words;
    // worst case: the carried tail completes one more block
    const uint64_t max_blocks = (r->nbits + ch.plan->n - 1) / ch.plan->n + 1;
    r->out_words = out_words_for(max_blocks * ch.plan->m);
    if ((!S->cfg.fake_executor && !out_host) || out_capacity_words < r->out_words) {
        delete r;
        return QEXT_E_NOSPACE;
    }
    if (request_bytes(*r) > S->arena.size()) {
        delete r;
        return QEXT_E_BUDGET;  // can never be admitted
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    ch.queue.push_back(r);
    S->arrivals.push_back(r);
    S->stats.submitted++;
    *request_id = r->id;
    S->cv.notify_all();
    return QEXT_OK;
}

int qext_server_poll(qext_server *S, qext_completion *out, uint32_t max, uint32_t *n) {
    if (!S || !n || (max && !out)) return QEXT_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    const uint32_t k = uint32_t(std::min<size_t>(max, S->completions.size()));
    for (uint32_t i = 0; i < k; ++i) out[i] = S->completions[i];
    S->completions.erase(S->completions.begin(), S->completions.begin() + k);
    *n = k;
    return QEXT_OK;
}

int qext_server_drain(qext_server *S, double timeout_s) {
    if (!S) return QEXT_E_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->stats.completed < S->stats.submitted) {
        if (S->cv.wait_until(lk, until) == std::cv_status::timeout && S->stats.completed < S->stats.submitted)
            return QEXT_E_TIMEOUT;
    }
    return QEXT_OK;
}

int qext_server_get_stats(qext_server *S, qext_server_stats *st) {
    if (!S || !st) return QEXT_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->stats;
    st->bytes_in_use = S->arena.used();
    st->peak_bytes = S->arena.peak();
    st->budget_bytes = S->arena.size();
    return QEXT_OK;
}

}  // extern "C"
